/*
 * pamc_oracle.c -- plain single-threaded CPU restatement of augmented PAMC.
 *
 * TEST INFRASTRUCTURE ONLY (see pamc_oracle.h).  Built with
 * -ffp-contract=off so that every floating-point operation is exactly the one
 * written; the only fused operation is the explicit fma() of det_exp.
 *
 * Conventions (readings of the paper where it is silent or ambiguous):
 *  - Ising energy H(s) = -sum_{i<j} J_ij s_i s_j (Sec. I; each pair once),
 *    Max-Cut couplings J = -w, so cut = (W - H)/2 with W = sum_{i<j} w_ij.
 *  - Potts energy (Eq. 6) with the same pair convention and J = -w, so the
 *    three-cut is (W - E)/2 as well.
 */
#include "pamc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4.1, "Philox").           */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    /* multipliers and Weyl key increments as published for Philox-4x32 */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void orc_draw4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------ */
/* Deterministic exp (Cody & Waite range reduction + Taylor series).   */
/* ------------------------------------------------------------------ */
/* ln 2 split: LN2_HI has 32 significant bits so k*LN2_HI is exact,
 * LN2_LO = ln 2 - LN2_HI rounded to binary64; 1/n! rounded to binary64. */
static const double ORC_LN2_HI = 0x1.62e42fee00000p-1;
static const double ORC_LN2_LO = 0x1.a39ef35793c76p-33;
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;
static const double ORC_INV_FACT[14] = {
    1.0, 1.0, 0x1.0000000000000p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5,
    0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
    0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26, 0x1.1eed8eff8d898p-29,
    0x1.6124613a86d09p-33};

double orc_det_exp(double x) {
    if (x != x) return x;
    if (x > 709.0) return INFINITY;
    if (x < -707.0) return 0.0;
    /* k = nearest integer to x / ln 2 */
    double kd = floor(x * ORC_INV_LN2 + 0.5);
    /* r = x - k ln2 in two exact-product steps */
    double r = fma(-kd, ORC_LN2_HI, x);
    r = fma(-kd, ORC_LN2_LO, r);
    /* e^r = sum_{i=0}^{13} r^i / i!  by Horner's rule */
    double p = ORC_INV_FACT[13];
    for (int i = 12; i >= 0; --i) p = fma(p, r, ORC_INV_FACT[i]);
    return ldexp(p, (int)kd);
}

uint64_t orc_round_nonneg(double x) {
    double f = floor(x);
    double frac = x - f;
    uint64_t v = (uint64_t)f;
    if (frac >= 0.5) v += 1;
    return v;
}

static const double ORC_TWO32 = 4294967296.0;

uint64_t orc_thr_heatbath(double beta, int64_t h) {
    /* P(s=+1) = (1 + tanh(beta h))/2 = 1/(1 + e^{-2 beta h})  (Eq. 4) */
    double x = -2.0 * beta * (double)h;
    double e = orc_det_exp(x);
    double p = 1.0 / (1.0 + e);
    return orc_round_nonneg(p * ORC_TWO32);
}

uint64_t orc_thr_metropolis(double beta, int64_t dE) {
    if (dE <= 0) return (uint64_t)1 << 32;
    double e = orc_det_exp(-(beta * (double)dE));
    return orc_round_nonneg(e * ORC_TWO32);
}

uint64_t orc_thr_potts_b1(double beta, int64_t a, int64_t b) {
    double ea = orc_det_exp(beta * (double)a);
    double eb = orc_det_exp(beta * (double)b);
    double den = (1.0 + ea) + eb;
    return orc_round_nonneg((1.0 / den) * ORC_TWO32);
}

uint64_t orc_thr_potts_b2(double beta, int64_t c) {
    double ec = orc_det_exp(beta * (double)c);
    return orc_round_nonneg((1.0 / (1.0 + ec)) * ORC_TWO32);
}

/* ------------------------------------------------------------------ */
/* Randomised sweep order (Sec. III.A, last sentence before Sec. III.B). */
/* ------------------------------------------------------------------ */
/* Reading: the paper asks only for a random order.  One order per
 * (step, sweep), shared by every replica: the indices sorted by a 32-bit
 * PERM draw, the index breaking ties. */
typedef struct { uint32_t key; int32_t idx; } orc_keyed;

static int orc_cmp_keyed(const void *a, const void *b) {
    const orc_keyed *x = (const orc_keyed *)a, *y = (const orc_keyed *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

void orc_permutation(int32_t n, uint64_t seed, int32_t t, int32_t sweep, int32_t *perm) {
    orc_keyed *a = (orc_keyed *)malloc(sizeof(orc_keyed) * (size_t)(n > 0 ? n : 1));
    for (int32_t k = 0; k < n; ++k) {
        uint32_t u[4];
        orc_draw4(seed, (uint32_t)k, (uint32_t)sweep, (uint32_t)t, (uint32_t)ORC_TAG_PERM << 24, u);
        a[k].key = u[0];
        a[k].idx = k;
    }
    qsort(a, (size_t)n, sizeof(orc_keyed), orc_cmp_keyed);
    for (int32_t p = 0; p < n; ++p) perm[p] = a[p].idx;
    free(a);
}

/* ------------------------------------------------------------------ */
/* Systematic resampling (Eq. 1-2; Fig. 2).                            */
/* ------------------------------------------------------------------ */
/* Readings: tau_j are expected copy numbers summing to R (Eq. 1 as printed
 * normalises them to 1, which contradicts Q = (1/R) sum of Eq. 2); the
 * population size stays R and the copies are drawn by systematic resampling
 * over the inclusive prefix of integer weights; the paper gives no energy
 * shift, so the weights are taken relative to E_min (cooling) or E_max
 * (reheating), which keeps exp from underflowing and gives the reference
 * replica weight 1. */
int orc_resample(int32_t R, const int64_t *E, double delta, double escale, uint64_t seed,
                 int32_t t, int32_t *parent, int32_t *count) {
    if (R <= 0) return -1;
    /* shift by the extreme energy so that the reference replica has weight 1 */
    int64_t emin = E[0], emax = E[0];
    for (int32_t r = 1; r < R; ++r) {
        if (E[r] < emin) emin = E[r];
        if (E[r] > emax) emax = E[r];
    }
    int lg = 0;
    while (((int64_t)1 << lg) < (int64_t)R) ++lg;
    int S = 62 - lg;
    double a = fabs(delta) * escale;
    uint64_t *C = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)R);
    uint64_t acc = 0;
    for (int32_t r = 0; r < R; ++r) {
        int64_t d = 0;
        if (delta > 0) d = E[r] - emin;
        else if (delta < 0) d = emax - E[r];
        double w = orc_det_exp(-(a * (double)d));
        uint64_t q = (uint64_t)floor(ldexp(w, S));
        acc += q;
        C[r] = acc;              /* inclusive prefix sum */
    }
    uint64_t T = acc;
    uint32_t u[4];
    orc_draw4(seed, 0u, 0u, (uint32_t)t, (uint32_t)ORC_TAG_RESAMPLE << 24, u);
    uint64_t v = ((uint64_t)u[1] << 32) | (uint64_t)u[0];
    uint64_t U = (uint64_t)(((unsigned __int128)v * (unsigned __int128)T) >> 64);
    for (int32_t j = 0; j < R; ++j) count[j] = 0;
    int32_t j = 0;
    for (int32_t m = 0; m < R; ++m) {
        unsigned __int128 pos = (unsigned __int128)m * T + U;
        /* smallest j with pos < R * C_j */
        while ((unsigned __int128)R * C[j] <= pos) ++j;
        parent[m] = j;
        count[j] += 1;
    }
    free(C);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Instance and state                                                  */
/* ------------------------------------------------------------------ */
struct orc_state {
    orc_params p;
    int32_t n;
    int32_t *rp, *col, *J;
    int64_t W;
    double dbeta;
    int8_t *s;         /* R*n */
    int32_t *h;        /* Ising R*n ; Potts R*n*3 */
    int64_t *E;        /* R */
    int8_t *s_tmp;
    int32_t *h_tmp;
    int64_t *E_tmp;
    int32_t *parent, *count;
    int32_t t, z, cycle, cooldown, enable_cm, done, ncm_last;
    int64_t ncm_flipped, ncm_dE_max;
    double beta, delta;
    int64_t mstar;
    int8_t *best;
    int64_t hist[ORC_HIST_MAX];
    int32_t hist_len;
    int32_t *ncm_targets;      /* slots of the last iteration's cluster move */
    int32_t n_ncm_targets;
    int64_t sweep_flips;       /* Ising: replica spins the sweeps changed */
    uint8_t *rmask;            /* sampled sweeps: sweep replica r iff rmask[r] */
    int8_t *r_spins;           /* sampled sweeps: the other replicas' results */
    int32_t own_lo, own_hi;    /* slots this state moves (NCM, sweeps); all R unless split */
    int32_t best_owned;        /* the last M* improvement came from an own slot */
};

static int32_t nf(const orc_state *st) { return st->p.kind == 1 ? st->p.K : 1; }

int64_t orc_energy_ising(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *J,
                         const int8_t *s) {
    int64_t E = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = col[e];
            if (i < j) E -= (int64_t)J[e] * s[i] * s[j];
        }
    return E;
}

int64_t orc_energy_potts(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *J,
                         const int8_t *sg) {
    int64_t E = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = col[e];
            if (i < j) E -= (int64_t)J[e] * (2 * (sg[i] == sg[j]) - 1);
        }
    return E;
}

/* fields from the definition: Ising h_k = sum_j J_kj s_j (Eq. 3);
 * Potts syn_c(k) = sum_j J_kj delta(sigma_j, c) (Eq. 7) */
static void orc_fields_replica(const orc_state *st, const int8_t *s, int32_t *h) {
    int32_t n = st->n;
    if (st->p.kind == 0) {
        for (int32_t k = 0; k < n; ++k) {
            int32_t acc = 0;
            for (int32_t e = st->rp[k]; e < st->rp[k + 1]; ++e) acc += st->J[e] * s[st->col[e]];
            h[k] = acc;
        }
    } else {
        int32_t K = st->p.K;
        for (int32_t k = 0; k < n; ++k) {
            int32_t *a = h + (size_t)K * k;
            for (int32_t c = 0; c < K; ++c) a[c] = 0;
            for (int32_t e = st->rp[k]; e < st->rp[k + 1]; ++e) a[s[st->col[e]]] += st->J[e];
        }
    }
}

static int64_t orc_energy_replica(const orc_state *st, const int8_t *s) {
    return st->p.kind == 0 ? orc_energy_ising(st->n, st->rp, st->col, st->J, s)
                           : orc_energy_potts(st->n, st->rp, st->col, st->J, s);
}

static void orc_refresh_replica(orc_state *st, int32_t r) {
    int32_t n = st->n;
    orc_fields_replica(st, st->s + (size_t)r * n, st->h + (size_t)r * n * nf(st));
    st->E[r] = orc_energy_replica(st, st->s + (size_t)r * n);
}

/* Random initial population (Algorithm 1, Initialization), keyed by step t.
 * Reading: a restart that resets the system draws a fresh population keyed
 * by the index of the step that starts from it (t + 1 for a restart decided
 * at the end of step t). */
static void orc_init_population(orc_state *st, int32_t t) {
    int32_t n = st->n, R = st->p.R;
    for (int32_t r = 0; r < R; ++r) {
        for (int32_t i = 0; i < n; ++i) {
            uint32_t u[4];
            orc_draw4(st->p.seed, (uint32_t)i, 0u, (uint32_t)t,
                      ((uint32_t)ORC_TAG_INIT << 24) | (uint32_t)(r >> 2), u);
            uint32_t x = u[r & 3];
            int8_t v;
            if (st->p.kind == 0) v = (x >> 31) ? 1 : -1;
            else v = (int8_t)(((uint64_t)x * (uint64_t)st->p.K) >> 32);
            st->s[(size_t)r * n + i] = v;
        }
        orc_refresh_replica(st, r);
    }
}

orc_state *orc_create(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                      const orc_params *p) {
    if (n <= 0 || !rp || !p || p->R <= 0 || p->sweeps < 0 || p->steps <= 0) return NULL;
    if (p->kind != 0 && p->kind != 1) return NULL;
    if (p->kind == 1 && !((p->rule == 0 && p->K == 3) || (p->rule == 2 && p->K >= 2 && p->K <= 8)))
        return NULL;
    if (p->kind == 1 && p->rule == 2 && !(p->gamma >= 0.0)) return NULL;
    if (rp[0] != 0) return NULL;
    int32_t nnz = rp[n];
    for (int32_t i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return NULL;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = col[e];
            if (j < 0 || j >= n || j == i) return NULL;
            /* symmetric: find (j, i) with the same weight */
            int found = 0;
            for (int32_t f = rp[j]; f < rp[j + 1]; ++f)
                if (col[f] == i && w[f] == w[e]) { found = 1; break; }
            if (!found) return NULL;
        }
    }
    orc_state *st = (orc_state *)calloc(1, sizeof(orc_state));
    st->p = *p;
    st->n = n;
    st->rp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    st->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    st->J = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    memcpy(st->rp, rp, sizeof(int32_t) * (size_t)(n + 1));
    int64_t wsum = 0;
    for (int32_t e = 0; e < nnz; ++e) {
        st->col[e] = col[e];
        st->J[e] = -w[e];        /* Max-Cut -> Ising couplings */
        wsum += w[e];
    }
    st->W = wsum / 2;            /* each unordered pair appears twice */
    int32_t R = p->R;
    size_t sn = (size_t)R * n;
    st->s = (int8_t *)malloc(sn);
    st->s_tmp = (int8_t *)malloc(sn);
    st->h = (int32_t *)malloc(sizeof(int32_t) * sn * nf(st));
    st->h_tmp = (int32_t *)malloc(sizeof(int32_t) * sn * nf(st));
    st->E = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    st->E_tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    st->parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
    st->count = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
    st->best = (int8_t *)calloc((size_t)n, 1);
    st->ncm_targets = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
    st->n_ncm_targets = 0;
    st->rmask = NULL;
    st->r_spins = NULL;
    st->own_lo = 0;
    st->own_hi = R;
    st->best_owned = 1;
    st->dbeta = p->steps > 1 ? (p->beta1 - p->beta0) / (double)(p->steps - 1) : 0.0;
    st->t = 0; st->z = 1; st->cycle = 0; st->cooldown = 0; st->enable_cm = 0; st->done = 0;
    st->beta = p->beta0; st->delta = st->dbeta;
    st->mstar = INT64_MIN;
    st->hist_len = 0;
    for (int32_t r = 0; r < R; ++r) { st->parent[r] = r; st->count[r] = 1; }
    orc_init_population(st, 0);
    return st;
}

void orc_destroy(orc_state *st) {
    if (!st) return;
    free(st->rp); free(st->col); free(st->J); free(st->s); free(st->s_tmp); free(st->h);
    free(st->h_tmp); free(st->E); free(st->E_tmp); free(st->parent); free(st->count);
    free(st->best); free(st->ncm_targets); free(st->rmask); free(st->r_spins); free(st);
}

/* ------------------------------------------------------------------ */
/* Single-spin sweeps                                                  */
/* ------------------------------------------------------------------ */
/* Ising, Eq. 3-4: visit the spins in the sweep's order; heat-bath sets
 * s_k = +1 iff u < T(h_k); Metropolis flips iff u < T_M(2 s_k h_k).  On a
 * change the neighbours' fields move by 2 s_k^new J_jk.  Readings: the pair
 * sum runs over i < j, so Eq. 4 is the exact conditional; the draw u / 2^32
 * plays r, and u == T (the tie of sgn(0)) gives -1. */
static void orc_sweep_ising(orc_state *st, int32_t r, const int32_t *perm, int32_t sweep) {
    int32_t n = st->n;
    int8_t *s = st->s + (size_t)r * n;
    int32_t *h = st->h + (size_t)r * n;
    for (int32_t p = 0; p < n; ++p) {
        int32_t k = perm[p];
        uint32_t u4[4];
        orc_draw4(st->p.seed, (uint32_t)k, (uint32_t)sweep, (uint32_t)st->t,
                  ((uint32_t)ORC_TAG_FLIP << 24) | (uint32_t)(r >> 2), u4);
        uint64_t u = u4[r & 3];
        int8_t old = s[k], nw;
        if (st->p.rule == 0) {
            nw = (u < orc_thr_heatbath(st->beta, h[k])) ? 1 : -1;
        } else {
            int64_t dE = 2 * (int64_t)old * h[k];
            nw = (u < orc_thr_metropolis(st->beta, dE)) ? (int8_t)-old : old;
        }
        if (nw != old) {
            st->sweep_flips += 1;
            st->E[r] += 2 * (int64_t)old * h[k];
            s[k] = nw;
            for (int32_t e = st->rp[k]; e < st->rp[k + 1]; ++e) h[st->col[e]] += 2 * nw * st->J[e];
        }
    }
}

/* Potts K=3 with the cascaded sampler (Suppl. S3): label 0 with
 * P = 1/(1+e^{beta(syn1-syn0)}+e^{beta(syn2-syn0)}) from draw u0, else label 1
 * with P = 1/(1+e^{beta(syn2-syn1)}) from draw u1, else label 2. */
static void orc_sweep_potts(orc_state *st, int32_t r, const int32_t *perm, int32_t sweep) {
    int32_t n = st->n;
    int8_t *s = st->s + (size_t)r * n;
    int32_t *h = st->h + (size_t)r * n * 3;
    for (int32_t p = 0; p < n; ++p) {
        int32_t k = perm[p];
        uint32_t u4[4];
        orc_draw4(st->p.seed, (uint32_t)k, (uint32_t)sweep, (uint32_t)st->t,
                  ((uint32_t)ORC_TAG_FLIP << 24) | (uint32_t)(r >> 1), u4);
        uint64_t u0 = u4[2 * (r & 1)], u1 = u4[2 * (r & 1) + 1];
        int32_t s0 = h[3 * k], s1 = h[3 * k + 1], s2 = h[3 * k + 2];
        int8_t old = s[k], nw;
        if (u0 < orc_thr_potts_b1(st->beta, (int64_t)s1 - s0, (int64_t)s2 - s0)) nw = 0;
        else if (u1 < orc_thr_potts_b2(st->beta, (int64_t)s2 - s1)) nw = 1;
        else nw = 2;
        if (nw != old) {
            st->E[r] += -2 * ((int64_t)h[3 * k + nw] - h[3 * k + old]);
            s[k] = nw;
            for (int32_t e = st->rp[k]; e < st->rp[k + 1]; ++e) {
                int32_t j = st->col[e];
                h[3 * j + old] -= st->J[e];
                h[3 * j + nw] += st->J[e];
            }
        }
    }
}

int32_t orc_softmax_pick(int32_t K, const int32_t *syn, double beta, double gamma, const uint32_t *u) {
    int32_t smax = syn[0];
    for (int32_t c = 1; c < K; ++c)
        if (syn[c] > smax) smax = syn[c];
    float e[8];
    float S = 0.0f;
    for (int32_t c = 0; c < K; ++c) {
        e[c] = (float)orc_det_exp(-(beta * (double)(smax - syn[c])));
        S = S + e[c];
    }
    const float g = (float)gamma;
    int32_t best = 0;
    float vbest = 0.0f;
    for (int32_t c = 0; c < K; ++c) {
        const float P = e[c] / S;
        const float U = (float)u[c] * 0x1p-32f;
        const float v = P - g * U;
        if (c == 0 || v > vbest) { vbest = v; best = c; }
    }
    return best;
}

/* Potts with K labels and the softmax noisy-argmax update (Sec. III.F, Eq. 8-9):
 * the draws of replica r at vertex k are words c mod 4 of Philox counters
 * (k, sweep, t, FLIP<<24 | (r * ceil(K/4) + c/4)), c = 0..K-1. */
static void orc_sweep_potts_softmax(orc_state *st, int32_t r, const int32_t *perm, int32_t sweep) {
    int32_t n = st->n, K = st->p.K, nb = (K + 3) / 4;
    int8_t *s = st->s + (size_t)r * n;
    int32_t *h = st->h + (size_t)r * n * K;
    for (int32_t p = 0; p < n; ++p) {
        int32_t k = perm[p];
        uint32_t u[8];
        for (int32_t b = 0; b < nb; ++b) {
            uint32_t u4[4];
            orc_draw4(st->p.seed, (uint32_t)k, (uint32_t)sweep, (uint32_t)st->t,
                      ((uint32_t)ORC_TAG_FLIP << 24) | (uint32_t)(r * nb + b), u4);
            for (int32_t q = 0; q < 4 && 4 * b + q < K; ++q) u[4 * b + q] = u4[q];
        }
        int8_t old = s[k];
        int8_t nw = (int8_t)orc_softmax_pick(K, h + (size_t)K * k, st->beta, st->p.gamma, u);
        if (nw != old) {
            st->E[r] += -2 * ((int64_t)h[(size_t)K * k + nw] - h[(size_t)K * k + old]);
            s[k] = nw;
            for (int32_t e = st->rp[k]; e < st->rp[k + 1]; ++e) {
                int32_t j = st->col[e];
                h[(size_t)K * j + old] -= st->J[e];
                h[(size_t)K * j + nw] += st->J[e];
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Non-local cluster move (Sec. III.C, NCM bullet)                      */
/* ------------------------------------------------------------------ */
/* Readings: the paper fixes neither the number of greedy MIS trials nor the
 * number of low-energy replicas that take the move; both are parameters.
 * Trial a orders the iso-sites by an NCM draw keyed (site, a, step, replica);
 * the largest set wins, ties to the earliest trial. */
int32_t orc_ncm_replica(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *J,
                        int8_t *s, int32_t *h, int32_t mis_trials, uint64_t seed, int32_t t,
                        int32_t r) {
    /* iso-sites: local field exactly zero, so a lone flip costs nothing */
    int32_t niso = 0;
    int32_t *iso = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t k = 0; k < n; ++k)
        if (h[k] == 0) iso[niso++] = k;
    orc_keyed *ord = (orc_keyed *)malloc(sizeof(orc_keyed) * (size_t)(niso > 0 ? niso : 1));
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)(niso > 0 ? niso : 1));
    int32_t *bestsel = (int32_t *)malloc(sizeof(int32_t) * (size_t)(niso > 0 ? niso : 1));
    int8_t *taken = (int8_t *)calloc((size_t)n, 1);
    int32_t nbest = -1;
    for (int32_t a = 0; a < mis_trials; ++a) {
        /* random permutation of the iso-sites */
        for (int32_t i = 0; i < niso; ++i) {
            uint32_t u[4];
            orc_draw4(seed, (uint32_t)iso[i], (uint32_t)a, (uint32_t)t,
                      ((uint32_t)ORC_TAG_NCM << 24) | (uint32_t)r, u);
            ord[i].key = u[0];
            ord[i].idx = iso[i];
        }
        qsort(ord, (size_t)niso, sizeof(orc_keyed), orc_cmp_keyed);
        /* greedy: take a site if it has zero coupling to every site taken */
        int32_t nsel = 0;
        for (int32_t i = 0; i < niso; ++i) {
            int32_t k = ord[i].idx, ok = 1;
            for (int32_t e = rp[k]; e < rp[k + 1] && ok; ++e)
                if (taken[col[e]] && J[e] != 0) ok = 0;
            if (ok) { sel[nsel++] = k; taken[k] = 1; }
        }
        for (int32_t q = 0; q < nsel; ++q) taken[sel[q]] = 0;
        if (nsel > nbest) {      /* strictly larger: ties keep the earliest trial */
            nbest = nsel;
            memcpy(bestsel, sel, sizeof(int32_t) * (size_t)nsel);
        }
    }
    if (nbest < 0) nbest = 0;
    for (int32_t q = 0; q < nbest; ++q) {
        int32_t k = bestsel[q];
        s[k] = (int8_t)-s[k];
        for (int32_t e = rp[k]; e < rp[k + 1]; ++e) h[col[e]] += 2 * s[k] * J[e];
    }
    free(iso); free(ord); free(sel); free(bestsel); free(taken);
    return nbest;
}

/* n_top replicas with the lowest (energy, index) */
static int64_t *orc_sort_E;
static int orc_cmp_energy_idx(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (orc_sort_E[x] != orc_sort_E[y]) return orc_sort_E[x] < orc_sort_E[y] ? -1 : 1;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int32_t orc_distinct_last(const int64_t *hist, int32_t len, int32_t w) {
    if (w > len) w = len;
    int32_t d = 0;
    for (int32_t i = len - w; i < len; ++i) {
        int seen = 0;
        for (int32_t q = len - w; q < i; ++q)
            if (hist[q] == hist[i]) { seen = 1; break; }
        if (!seen) ++d;
    }
    return d;
}

/* ------------------------------------------------------------------ */
/* Adaptive temperature control and restart (Algorithm 1, after the    */
/* sweeps; the stagnation rule of Sec. III.C, second bullet).           */
/* ------------------------------------------------------------------ */
/* Readings: where the branches of Algorithm 1 and the text disagree the text
 * is taken -- progress keeps cooling; a stagnant short window alone reverses
 * the update only above beta0, and the listing's early exit changes nothing;
 * control runs once the history holds win_long values; a restart clears the
 * history and returns to beta0; beta advances by repeated addition. */
int orc_control(orc_ctl *c, const orc_params *p, double dbeta, int64_t mstar) {
    /* record M* in the recent-progress history (the last win_long values) */
    int32_t hl = p->win_long > p->win_short ? p->win_long : p->win_short;
    if (hl > ORC_HIST_MAX) hl = ORC_HIST_MAX;
    if (hl > 0) {
        if (c->hist_len == hl) {
            memmove(c->hist, c->hist + 1, sizeof(int64_t) * (size_t)(hl - 1));
            c->hist_len = hl - 1;
        }
        c->hist[c->hist_len++] = mstar;
    }
    if (p->stagnation && c->cooldown == 0 && hl > 0 && c->hist_len >= hl) {
        int32_t ds = orc_distinct_last(c->hist, c->hist_len, p->win_short);
        int32_t dl = orc_distinct_last(c->hist, c->hist_len, p->win_long);
        if (ds <= p->max_distinct_short && dl <= p->max_distinct_long) {
            /* both windows stagnant: reheat and arm the cluster move */
            c->beta = p->reheat_factor * c->beta;
            c->delta = dbeta;
            c->enable_cm = 1;
        } else if (ds <= p->max_distinct_short) {
            /* short window stagnant only: reverse the beta update */
            if (c->beta > p->beta0) c->delta = -dbeta;
        } else {
            /* progress: usual cooling direction */
            c->delta = dbeta;
        }
    }
    if (p->z_rst > 0 && c->z >= p->z_rst) {
        c->cycle += 1;
        c->z = 1;
        c->beta = p->beta0;
        c->delta = dbeta;
        c->enable_cm = 0;
        c->cooldown = 0;
        c->hist_len = 0;
        return 1;
    }
    c->z += 1;
    c->beta = c->beta + c->delta;
    if (c->cooldown > 0) c->cooldown -= 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* One iteration of Algorithm 1                                        */
/* ------------------------------------------------------------------ */
/* Algorithm 1, one iteration, in its three parts: the population step
 * (resampling at the new beta, then the cluster moves), the S sweeps, and
 * M* with the controller. */
void orc_iter_population(orc_state *st) {
    int32_t n = st->n, R = st->p.R, F = nf(st);
    /* Reading: the Potts update follows Eq. 8 literally (P ~ e^{beta syn_k}),
     * which samples e^{-(beta/2) E} with E of Eq. 6, so the reweighting uses
     * half the energy for Potts. */
    double escale = st->p.kind == 1 ? 0.5 : 1.0;
    st->ncm_last = 0;
    st->n_ncm_targets = 0;
    for (int32_t r = 0; r < R; ++r) { st->parent[r] = r; st->count[r] = 1; }
    if (st->z > 1) {
        if (st->p.resample) {
            orc_resample(R, st->E, st->delta, escale, st->p.seed, st->t, st->parent, st->count);
            for (int32_t m = 0; m < R; ++m) {
                int32_t j = st->parent[m];
                memcpy(st->s_tmp + (size_t)m * n, st->s + (size_t)j * n, (size_t)n);
                memcpy(st->h_tmp + (size_t)m * n * F, st->h + (size_t)j * n * F,
                       sizeof(int32_t) * (size_t)n * F);
                st->E_tmp[m] = st->E[j];
            }
            memcpy(st->s, st->s_tmp, (size_t)R * n);
            memcpy(st->h, st->h_tmp, sizeof(int32_t) * (size_t)R * n * F);
            memcpy(st->E, st->E_tmp, sizeof(int64_t) * (size_t)R);
        }
        if (st->enable_cm && st->cooldown == 0) {
            if (st->p.kind == 0) {
                int32_t ntop = st->p.n_top < R ? st->p.n_top : R;
                int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
                for (int32_t r = 0; r < R; ++r) idx[r] = r;
                orc_sort_E = st->E;
                qsort(idx, (size_t)R, sizeof(int32_t), orc_cmp_energy_idx);
                for (int32_t q = 0; q < ntop; ++q) {
                    int32_t r = idx[q];
                    st->ncm_targets[st->n_ncm_targets++] = r;
                    if (r < st->own_lo || r >= st->own_hi) continue;   /* another process's slot */
                    int64_t before = st->E[r];
                    st->ncm_flipped += orc_ncm_replica(n, st->rp, st->col, st->J,
                                                       st->s + (size_t)r * n, st->h + (size_t)r * n,
                                                       st->p.mis_trials, st->p.seed, st->t, r);
                    /* energy from the definition: the move must leave it unchanged */
                    st->E[r] = orc_energy_replica(st, st->s + (size_t)r * n);
                    int64_t d = st->E[r] - before;
                    if (d < 0) d = -d;
                    if (d > st->ncm_dE_max) st->ncm_dE_max = d;
                }
                free(idx);
            }
            st->ncm_last = 1;
            st->enable_cm = 0;
            st->cooldown = st->p.cooldown_tau;
        }
    }
}

void orc_iter_sweeps(orc_state *st) {
    int32_t n = st->n, R = st->p.R;
    /* S sweeps at the current beta */
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t sw = 0; sw < st->p.sweeps; ++sw) {
        orc_permutation(n, st->p.seed, st->t, sw, perm);
        for (int32_t r = st->own_lo; r < st->own_hi; ++r) {
            if (st->rmask && !st->rmask[r]) continue;
            if (st->p.kind == 0) orc_sweep_ising(st, r, perm, sw);
            else if (st->p.rule == 2) orc_sweep_potts_softmax(st, r, perm, sw);
            else orc_sweep_potts(st, r, perm, sw);
        }
    }
    free(perm);
    /* sampled sweeps: the replicas outside the sample take the results given */
    if (st->rmask)
        for (int32_t r = 0; r < R; ++r)
            if (!st->rmask[r]) {
                memcpy(st->s + (size_t)r * n, st->r_spins + (size_t)r * n, (size_t)n);
                orc_refresh_replica(st, r);
            }
}

void orc_iter_control(orc_state *st) {
    int32_t n = st->n, R = st->p.R;
    /* M* <- max(M*, max Cut(P)); cut = (W - E)/2 */
    int32_t rbest = 0;
    for (int32_t r = 1; r < R; ++r)
        if (st->E[r] < st->E[rbest]) rbest = r;
    int64_t cut = (st->W - st->E[rbest]) / 2;
    if (cut > st->mstar) {
        st->mstar = cut;
        st->best_owned = rbest >= st->own_lo && rbest < st->own_hi;
        if (st->best_owned) memcpy(st->best, st->s + (size_t)rbest * n, (size_t)n);
    }
    orc_ctl c;
    c.z = st->z; c.cycle = st->cycle; c.cooldown = st->cooldown; c.enable_cm = st->enable_cm;
    c.hist_len = st->hist_len; c.beta = st->beta; c.delta = st->delta;
    memcpy(c.hist, st->hist, sizeof(int64_t) * (size_t)st->hist_len);
    int restart = orc_control(&c, &st->p, st->dbeta, st->mstar);
    st->z = c.z; st->cycle = c.cycle; st->cooldown = c.cooldown; st->enable_cm = c.enable_cm;
    st->hist_len = c.hist_len; st->beta = c.beta; st->delta = c.delta;
    memcpy(st->hist, c.hist, sizeof(int64_t) * (size_t)c.hist_len);
    if (restart && st->p.restart_reinit) orc_init_population(st, st->t + 1);
    st->t += 1;
    if (st->p.target_cut >= 0 && st->mstar >= st->p.target_cut) st->done = 1;
}

static void orc_iteration(orc_state *st) {
    orc_iter_population(st);
    orc_iter_sweeps(st);
    orc_iter_control(st);
}

int32_t orc_step(orc_state *st, int32_t nsteps) {
    int32_t ran = 0;
    for (int32_t i = 0; i < nsteps && !st->done; ++i) {
        orc_iteration(st);
        ++ran;
    }
    return ran;
}

/* ------------------------------------------------------------------ */
/* Accessors                                                           */
/* ------------------------------------------------------------------ */
void orc_get_spins(const orc_state *st, int8_t *out) { memcpy(out, st->s, (size_t)st->p.R * st->n); }
void orc_get_fields(const orc_state *st, int32_t *out) {
    memcpy(out, st->h, sizeof(int32_t) * (size_t)st->p.R * st->n * nf(st));
}
void orc_get_energy(const orc_state *st, int64_t *out) { memcpy(out, st->E, sizeof(int64_t) * (size_t)st->p.R); }
void orc_get_parents(const orc_state *st, int32_t *parent, int32_t *count) {
    memcpy(parent, st->parent, sizeof(int32_t) * (size_t)st->p.R);
    memcpy(count, st->count, sizeof(int32_t) * (size_t)st->p.R);
}
void orc_get_best(const orc_state *st, int64_t *mstar, int8_t *spins) {
    *mstar = st->mstar;
    int32_t n = st->n;
    if (st->p.kind == 0) {
        int8_t f = st->best[0] < 0 ? -1 : 1;   /* canonical: spin 0 is +1 */
        for (int32_t i = 0; i < n; ++i) spins[i] = (int8_t)(st->best[i] * f);
    } else {
        int8_t map[8] = {-1, -1, -1, -1, -1, -1, -1, -1};   /* labels renamed in order of first use */
        int8_t next = 0;
        for (int32_t i = 0; i < n; ++i) {
            int8_t c = st->best[i];
            if (map[c] < 0) map[c] = next++;
            spins[i] = map[c];
        }
    }
}
void orc_get_ctl(const orc_state *st, int64_t *iv, double *dv) {
    iv[0] = st->t; iv[1] = st->z; iv[2] = st->cycle; iv[3] = st->cooldown;
    iv[4] = st->enable_cm; iv[5] = st->done; iv[6] = st->ncm_last; iv[7] = st->hist_len;
    iv[8] = st->ncm_flipped; iv[9] = st->ncm_dE_max;
    dv[0] = st->beta; dv[1] = st->delta;
}
int64_t orc_weight_sum(const orc_state *st) { return st->W; }
void orc_set_spins(orc_state *st, const int8_t *spins) {
    memcpy(st->s, spins, (size_t)st->p.R * st->n);
    for (int32_t r = 0; r < st->p.R; ++r) orc_refresh_replica(st, r);
}

void orc_set_state(orc_state *st, int32_t t, const orc_ctl *ctl, int64_t mstar, const int8_t *best,
                   const int8_t *spins) {
    st->t = t;
    st->z = ctl->z; st->cycle = ctl->cycle; st->cooldown = ctl->cooldown; st->enable_cm = ctl->enable_cm;
    st->beta = ctl->beta; st->delta = ctl->delta;
    st->hist_len = ctl->hist_len;
    memcpy(st->hist, ctl->hist, sizeof(int64_t) * (size_t)ctl->hist_len);
    st->mstar = mstar;
    if (best) memcpy(st->best, best, (size_t)st->n);
    st->done = 0;
    st->ncm_last = 0;
    st->ncm_flipped = 0;
    st->ncm_dE_max = 0;
    st->n_ncm_targets = 0;
    orc_set_spins(st, spins);
}

void orc_set_sweep_replay(orc_state *st, const uint8_t *mask, const int8_t *spins_after) {
    free(st->rmask);
    free(st->r_spins);
    st->rmask = NULL;
    st->r_spins = NULL;
    if (!mask) return;
    size_t R = (size_t)st->p.R, sn = R * (size_t)st->n;
    st->rmask = (uint8_t *)malloc(R);
    st->r_spins = (int8_t *)malloc(sn);
    memcpy(st->rmask, mask, R);
    memcpy(st->r_spins, spins_after, sn);
}

void orc_get_ncm_targets(const orc_state *st, int32_t *targets, int32_t *count) {
    memcpy(targets, st->ncm_targets, sizeof(int32_t) * (size_t)st->n_ncm_targets);
    *count = st->n_ncm_targets;
}

void orc_get_history(const orc_state *st, int64_t *hist) {
    memcpy(hist, st->hist, sizeof(int64_t) * (size_t)st->hist_len);
}

int64_t orc_sweep_flips(const orc_state *st) { return st->sweep_flips; }

void orc_set_own(orc_state *st, int32_t lo, int32_t hi) {
    if (lo < 0) lo = 0;
    if (hi > st->p.R) hi = st->p.R;
    st->own_lo = lo;
    st->own_hi = hi < lo ? lo : hi;
}
void orc_set_energies(orc_state *st, const int64_t *E) {
    memcpy(st->E, E, sizeof(int64_t) * (size_t)st->p.R);
}
void orc_set_rows(orc_state *st, int32_t r0, int32_t count, const int8_t *rows) {
    for (int32_t i = 0; i < count; ++i) {
        int32_t r = r0 + i;
        if (r < 0 || r >= st->p.R) continue;
        memcpy(st->s + (size_t)r * st->n, rows + (size_t)i * st->n, (size_t)st->n);
        orc_refresh_replica(st, r);
    }
}
int32_t orc_best_owned(const orc_state *st) { return st->best_owned; }
