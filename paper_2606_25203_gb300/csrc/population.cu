// population.cu -- the population step and the controller of Algorithm 1:
//   k_tables   acceptance thresholds for the current beta (Eq. 4, Metropolis,
//              Suppl. S3), in binary64 with the deterministic exp;
//   k_weights  the binary64 resampling weights of Eq. 1 as 64-bit fixed-point
//              integers, spread over many CTAs;
//   k_prep     Boltzmann reweighting and resampling (Eq. 1-2) as systematic
//              resampling over an integer prefix scan of 64-bit fixed-point
//              weights, and selection of the NCM targets;
//   k_ncm      the energy-preserving non-local cluster move (Sec. III.C):
//              randomised greedy maximal independent sets of iso-sites;
//   k_control  M* / best configuration, the recent-progress history, the
//              adaptive temperature rule (Sec. III.C) and the restart.
// All state lives on the device so that an iteration never waits for the host.
#include <cstdlib>

#include "pamc_device.cuh"
#include "pamc_internal.h"

namespace pamc {

namespace {

// ---------------------------------------------------------------- tables
__device__ __forceinline__ void tables_ising_body(int rule, int32_t H, const DevCtl *__restrict__ ctl,
                                                  uint64_t *__restrict__ tab, int bid, int nb) {
    if (ctl->done) return;
    const double beta = ctl->beta;
    const int32_t n = 2 * H + 1;
    for (int32_t i = bid * blockDim.x + threadIdx.x; i < n; i += nb * blockDim.x) {
        const int32_t v = i - H;   // h (heat-bath) or s*h (Metropolis, dE = 2 s h)
        tab[i] = rule == 0 ? thr_heatbath(beta, v) : thr_metropolis(beta, 2 * (int64_t)v);
    }
}

// Batched tables: kTabBlocks CTAs per member.  Ising: the 2H+1 thresholds;
// Potts (cascaded sampler): T1 over (a, b) in [-2H, 2H]^2, then T2 over c, the
// same values as the single-instance kernel below.
constexpr int kTabBlocks = 8;

__global__ void k_tables_batched(const TabDesc *__restrict__ descs) {
    __shared__ double e_s[4 * 127 + 1];
    const TabDesc d = descs[blockIdx.x / kTabBlocks];
    const int part = blockIdx.x % kTabBlocks;
    if (d.ctl->t >= d.t_end || d.ctl->done) return;
    if (d.kind == 0) {
        tables_ising_body(d.rule, d.H, d.ctl, d.tab, part, kTabBlocks);
        return;
    }
    const double beta = d.ctl->beta;
    const int32_t H = d.H, W1 = 4 * H + 1;
    for (int32_t i = threadIdx.x; i < W1; i += blockDim.x)
        e_s[i] = det_exp(__dmul_rn(beta, (double)(i - 2 * H)));
    __syncthreads();
    const int32_t total = W1 * W1 + W1;
    for (int32_t i = part * blockDim.x + threadIdx.x; i < total; i += kTabBlocks * blockDim.x) {
        if (i < W1 * W1) {
            d.tab[i] = thr_potts_b1_from(e_s[i / W1], e_s[i % W1]);
        } else {
            const int32_t c = i - W1 * W1;
            d.tab[i] = thr_potts_b2(beta, (int64_t)(c - 2 * H));
        }
    }
}

// Softmax Potts: e(d) = (float) exp(-beta d) for d = max_m syn_m - syn_c in [0, 2H].
__global__ void k_tables_softmax(int32_t H, const DevCtl *__restrict__ ctl, float *__restrict__ tab) {
    if (ctl->done) return;
    const double beta = ctl->beta;
    for (int32_t d = threadIdx.x; d <= 2 * H; d += blockDim.x)
        tab[d] = __double2float_rn(det_exp(-__dmul_rn(beta, (double)d)));
}

__global__ void k_tables(int kind, int rule, int32_t H, const DevCtl *__restrict__ ctl,
                         uint64_t *__restrict__ tab) {
    if (ctl->done) return;
    const double beta = ctl->beta;
    if (kind == 0) {
        const int32_t n = 2 * H + 1;
        for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const int32_t v = i - H;   // h (heat-bath) or s*h (Metropolis, dE = 2 s h)
            tab[i] = rule == 0 ? thr_heatbath(beta, v) : thr_metropolis(beta, 2 * (int64_t)v);
        }
        return;
    }
    // Potts: T1 over (a, b) in [-2H, 2H]^2, then T2 over c in [-2H, 2H]
    extern __shared__ double e_s[];
    const int32_t W1 = 4 * H + 1;
    for (int32_t i = threadIdx.x; i < W1; i += blockDim.x)
        e_s[i] = det_exp(__dmul_rn(beta, (double)(i - 2 * H)));
    __syncthreads();
    const int32_t total = W1 * W1 + W1;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < W1 * W1) {
            const int32_t ia = i / W1, ib = i % W1;
            tab[i] = thr_potts_b1_from(e_s[ia], e_s[ib]);
        } else {
            const int32_t c = i - W1 * W1;
            tab[i] = thr_potts_b2(beta, (int64_t)(c - 2 * H));
        }
    }
}

// ---------------------------------------------------------------- block helpers
template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T *sbuf) {
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sbuf[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        T a = sbuf[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) a = op(a, sbuf[i]);
        sbuf[0] = a;
    }
    __syncthreads();
    const T r = sbuf[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- resampling
constexpr int kPrepThreads = 1024;
constexpr int kWeightThreads = 256;

// Integer resampling weights q_r = floor(2^S * w_r), w_r = exp(-|Delta| d_r)
// (Eq. 1, the one binary64 step), spread over ceil(R / 256) CTAs: binary64
// arithmetic runs at a small fraction of the integer rate, so R weights in a
// single CTA would keep one SM busy for tens of microseconds.  Every CTA
// reduces E_min / E_max over the whole population itself.  Writes nothing
// when the step does not resample.
__global__ void __launch_bounds__(kWeightThreads)
k_weights(int32_t R, int32_t kind, int32_t do_resample, const int64_t *__restrict__ E_src,
          const DevCtl *__restrict__ ctl, uint64_t *__restrict__ q, const long long *__restrict__ mm) {
    __shared__ long long red_ll[32];
    if (ctl->done || !(ctl->z > 1 && do_resample)) return;
    const double delta = ctl->delta;
    long long emin, emax;
    if (mm) {   // large populations: reduced once by k_minmax
        emin = mm[0];
        emax = mm[1];
    } else {
        long long lmin = LLONG_MAX, lmax = LLONG_MIN;
        for (int32_t r = threadIdx.x; r < R; r += blockDim.x) {
            lmin = min(lmin, (long long)E_src[r]);
            lmax = max(lmax, (long long)E_src[r]);
        }
        emin = block_reduce(lmin, [](long long a, long long b) { return a < b ? a : b; }, red_ll);
        emax = block_reduce(lmax, [](long long a, long long b) { return a > b ? a : b; }, red_ll);
    }
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int lg = 0;
    while ((1ll << lg) < (long long)R) ++lg;
    const int S = 62 - lg;
    const double a = __dmul_rn(fabs(delta), kind == 1 ? 0.5 : 1.0);
    long long d = 0;
    if (delta > 0) d = (long long)E_src[r] - emin;
    else if (delta < 0) d = emax - (long long)E_src[r];
    const double w = det_exp(-__dmul_rn(a, (double)d));
    q[r] = (uint64_t)floor(ldexp(w, S));
}

__device__ __forceinline__ void
prep_body(int32_t R, int32_t kind, int32_t do_resample, int32_t n_top, int32_t tau, uint32_t key0,
          uint32_t key1, const int64_t *__restrict__ E_src, DevCtl *__restrict__ ctl,
          int32_t *__restrict__ parent, int32_t *__restrict__ count, int32_t *__restrict__ ncm_idx,
          int32_t *__restrict__ targets, int32_t *__restrict__ fam, int32_t fam_reset,
          const uint64_t *__restrict__ qpre) {
    extern __shared__ __align__(16) unsigned char sm[];
    uint64_t *C = reinterpret_cast<uint64_t *>(sm);             // R prefix sums
    int32_t *cnt = reinterpret_cast<int32_t *>(sm + (size_t)R * 8);
    __shared__ long long red_ll[32];
    __shared__ unsigned long long red_u[32];
    if (ctl->done) return;
    const int32_t z = ctl->z;
    const int32_t t = ctl->t;
    const double delta = ctl->delta;
    const bool resampled = z > 1 && do_resample;
    const bool ncm = z > 1 && ctl->enable_cm && ctl->cooldown == 0;
    const bool restarted = ctl->restart != 0;
    __syncthreads();

    for (int32_t m = threadIdx.x; m < R; m += blockDim.x) { cnt[m] = 0; ncm_idx[m] = -1; }
    __syncthreads();
    if (resampled) {
        // shift by the extreme energy: the reference replica has weight 1
        // (the weights come precomputed by k_weights when qpre is given)
        long long lmin = LLONG_MAX, lmax = LLONG_MIN;
        if (!qpre) {
            for (int32_t r = threadIdx.x; r < R; r += blockDim.x) {
                lmin = min(lmin, (long long)E_src[r]);
                lmax = max(lmax, (long long)E_src[r]);
            }
        }
        const long long emin =
            qpre ? 0 : block_reduce(lmin, [](long long a, long long b) { return a < b ? a : b; }, red_ll);
        const long long emax =
            qpre ? 0 : block_reduce(lmax, [](long long a, long long b) { return a > b ? a : b; }, red_ll);
        int lg = 0;
        while ((1ll << lg) < (long long)R) ++lg;
        const int S = 62 - lg;
        const double a = __dmul_rn(fabs(delta), kind == 1 ? 0.5 : 1.0);
        // contiguous chunk per thread for the scan
        const int32_t per = (R + blockDim.x - 1) / blockDim.x;
        const int32_t lo = min(R, (int32_t)threadIdx.x * per), hi = min(R, lo + per);
        unsigned long long local = 0;
        for (int32_t r = lo; r < hi; ++r) {
            uint64_t q;
            if (qpre) {
                q = qpre[r];
            } else {
                long long d = 0;
                if (delta > 0) d = (long long)E_src[r] - emin;
                else if (delta < 0) d = emax - (long long)E_src[r];
                const double w = det_exp(-__dmul_rn(a, (double)d));
                q = (uint64_t)floor(ldexp(w, S));
            }
            local += q;
            C[r] = local;   // chunk-local inclusive prefix
        }
        // exclusive scan of the chunk totals across the block
        unsigned long long x = local;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) red_u[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned long long v = lane < (int)(blockDim.x >> 5) ? red_u[lane] : 0ull;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            red_u[lane] = v;   // inclusive warp totals
        }
        __syncthreads();
        const unsigned long long excl = (x - local) + (wid > 0 ? red_u[wid - 1] : 0ull);
        for (int32_t r = lo; r < hi; ++r) C[r] += excl;
        __syncthreads();
        const uint64_t T = C[R - 1];
        const u32x4 u = philox(0u, 0u, (uint32_t)t, kTagResample << 24, key0, key1);
        const uint64_t v = ((uint64_t)u.y << 32) | (uint64_t)u.x;
        const uint64_t U = __umul64hi(v, T);
        for (int32_t m = threadIdx.x; m < R; m += blockDim.x) {
            const unsigned __int128 pos = (unsigned __int128)m * T + U;
            int32_t lo2 = 0, hi2 = R - 1;   // smallest j with R*C_j > pos
            while (lo2 < hi2) {
                const int32_t mid = (lo2 + hi2) >> 1;
                if ((unsigned __int128)R * C[mid] > pos) hi2 = mid;
                else lo2 = mid + 1;
            }
            parent[m] = lo2;
            atomicAdd(&cnt[lo2], 1);
        }
    } else {
        for (int32_t m = threadIdx.x; m < R; m += blockDim.x) { parent[m] = m; cnt[m] = 1; }
    }
    __syncthreads();
    for (int32_t m = threadIdx.x; m < R; m += blockDim.x) count[m] = cnt[m];
    // lineage: slot m joins its parent's family (double-buffered by step
    // parity); a re-initialised population starts new families
    if (fam) {
        const int32_t *fs = fam + (size_t)(t & 1) * R;
        int32_t *fd = fam + (size_t)((t + 1) & 1) * R;
        for (int32_t m = threadIdx.x; m < R; m += blockDim.x)
            fd[m] = (fam_reset && restarted) ? m : fs[parent[m]];
    }

    if (ncm && kind == 0) {
        // targets: the n_top slots with the lowest (energy, slot index), by a
        // block-wide bitonic sort of (energy, slot) pairs over the next power
        // of two (padding sorts last); the counts above are already stored,
        // so the whole shared buffer is free for the keys
        const int32_t ntop = min(n_top, R);
        int32_t P2 = 1;
        while (P2 < R) P2 <<= 1;
        int64_t *Ek = reinterpret_cast<int64_t *>(C);
        int32_t *Mi = reinterpret_cast<int32_t *>(sm + (size_t)P2 * 8);
        __syncthreads();
        for (int32_t m = threadIdx.x; m < P2; m += blockDim.x) {
            Ek[m] = m < R ? (int64_t)E_src[parent[m]] : INT64_MAX;
            Mi[m] = m < R ? m : INT32_MAX;
        }
        __syncthreads();
        for (int32_t k = 2; k <= P2; k <<= 1) {
            for (int32_t j = k >> 1; j > 0; j >>= 1) {
                for (int32_t i = threadIdx.x; i < P2; i += blockDim.x) {
                    const int32_t l = i ^ j;
                    if (l > i) {
                        const int64_t ei = Ek[i], el = Ek[l];
                        const int32_t mi = Mi[i], ml = Mi[l];
                        const bool gt = ei > el || (ei == el && mi > ml);
                        if (gt == ((i & k) == 0)) {   // ascending where bit k of i is clear
                            Ek[i] = el; Ek[l] = ei;
                            Mi[i] = ml; Mi[l] = mi;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int32_t q = threadIdx.x; q < ntop; q += blockDim.x) {
            const int32_t m = Mi[q];
            targets[q] = m;
            ncm_idx[m] = q;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->resampled = resampled ? 1 : 0;
        ctl->ncm_active = ncm ? 1 : 0;
        ctl->ncm_last = ncm ? 1 : 0;
        if (ncm) { ctl->enable_cm = 0; ctl->cooldown = tau; }
    }
}

__global__ void __launch_bounds__(kPrepThreads)
k_prep(int32_t R, int32_t kind, int32_t do_resample, int32_t n_top, int32_t tau, uint32_t key0,
       uint32_t key1, const int64_t *__restrict__ E_src, DevCtl *__restrict__ ctl,
       int32_t *__restrict__ parent, int32_t *__restrict__ count, int32_t *__restrict__ ncm_idx,
       int32_t *__restrict__ targets, int32_t *__restrict__ fam, int32_t fam_reset,
       const uint64_t *__restrict__ qpre) {
    prep_body(R, kind, do_resample, n_top, tau, key0, key1, E_src, ctl, parent, count, ncm_idx, targets, fam,
              fam_reset, qpre);
}

__global__ void __launch_bounds__(kPrepThreads) k_prep_batched(const PrepDesc *__restrict__ descs) {
    const PrepDesc d = descs[blockIdx.x];
    const int32_t t = d.ctl->t;
    if (t >= d.t_end) return;
    prep_body(d.R, d.kind, d.do_resample, d.n_top, d.tau, d.key0, d.key1, d.en[t & 1], d.ctl, d.parent, d.count,
              d.ncm_idx, d.targets, d.fam, d.fam_reset, nullptr);
}

// ---------------------------------------------------------------- large populations
// R > kPrepOneCtaMaxR: the prefix sums live in device memory and the steps
// of prep_body run as separate kernels -- the same definitions (Eq. 1-2,
// systematic resampling by binary search over the integer prefix sums, the
// n_top lowest (energy, slot) NCM targets), so every result is the one a
// single CTA would give.
constexpr int kBigThreads = 1024;

__global__ void __launch_bounds__(kBigThreads)
k_minmax(int32_t R, int32_t do_resample, const int64_t *__restrict__ E, const DevCtl *__restrict__ ctl,
         long long *__restrict__ mm) {
    __shared__ long long red_ll[32];
    if (ctl->done || !(ctl->z > 1 && do_resample)) return;
    long long lmin = LLONG_MAX, lmax = LLONG_MIN;
    for (int32_t r = threadIdx.x; r < R; r += blockDim.x) {
        lmin = min(lmin, (long long)E[r]);
        lmax = max(lmax, (long long)E[r]);
    }
    const long long emin = block_reduce(lmin, [](long long a, long long b) { return a < b ? a : b; }, red_ll);
    const long long emax = block_reduce(lmax, [](long long a, long long b) { return a > b ? a : b; }, red_ll);
    if (threadIdx.x == 0) { mm[0] = emin; mm[1] = emax; }
}

// Inclusive prefix sums of the weights, in place: a contiguous chunk per
// thread, the chunk totals scanned across the block (one CTA).
__global__ void __launch_bounds__(kBigThreads)
k_scan_big(int32_t R, int32_t do_resample, uint64_t *__restrict__ q, const DevCtl *__restrict__ ctl) {
    __shared__ unsigned long long red_u[32];
    if (ctl->done || !(ctl->z > 1 && do_resample)) return;
    const int32_t per = (R + blockDim.x - 1) / blockDim.x;
    const int32_t lo = min(R, (int32_t)threadIdx.x * per), hi = min(R, lo + per);
    unsigned long long local = 0;
    for (int32_t r = lo; r < hi; ++r) {
        local += q[r];
        q[r] = local;
    }
    unsigned long long x = local;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) red_u[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long v = lane < (int)(blockDim.x >> 5) ? red_u[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        red_u[lane] = v;
    }
    __syncthreads();
    const unsigned long long excl = (x - local) + (wid > 0 ? red_u[wid - 1] : 0ull);
    for (int32_t r = lo; r < hi; ++r) q[r] += excl;
}

// Parent of every slot (binary search over the prefix sums C), copy counts
// (count zeroed beforehand), lineage and the NCM index reset: one thread per slot.
__global__ void __launch_bounds__(256)
k_parent_big(int32_t R, int32_t do_resample, uint32_t key0, uint32_t key1, const uint64_t *__restrict__ C,
             const DevCtl *__restrict__ ctl, int32_t *__restrict__ parent, int32_t *__restrict__ count,
             int32_t *__restrict__ ncm_idx, int32_t *__restrict__ fam, int32_t fam_reset) {
    if (ctl->done) return;
    const int32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= R) return;
    const int32_t t = ctl->t;
    const bool resampled = ctl->z > 1 && do_resample;
    ncm_idx[m] = -1;
    int32_t pm = m;
    if (resampled) {
        const uint64_t T = C[R - 1];
        const u32x4 u = philox(0u, 0u, (uint32_t)t, kTagResample << 24, key0, key1);
        const uint64_t v = ((uint64_t)u.y << 32) | (uint64_t)u.x;
        const uint64_t U = __umul64hi(v, T);
        const unsigned __int128 pos = (unsigned __int128)m * T + U;
        int32_t lo2 = 0, hi2 = R - 1;   // smallest j with R*C_j > pos
        while (lo2 < hi2) {
            const int32_t mid = (lo2 + hi2) >> 1;
            if ((unsigned __int128)R * C[mid] > pos) hi2 = mid;
            else lo2 = mid + 1;
        }
        pm = lo2;
        atomicAdd(&count[pm], 1);
    } else {
        count[m] = 1;
    }
    parent[m] = pm;
    if (fam) {
        const int32_t *fs = fam + (size_t)(t & 1) * R;
        int32_t *fd = fam + (size_t)((t + 1) & 1) * R;
        fd[m] = (fam_reset && ctl->restart != 0) ? m : fs[pm];
    }
}

// NCM targets of a large population (one CTA): the n_top slots of lowest
// (energy, slot).  The n_top-th smallest energy is found by a radix select
// over E - E_min (eight passes of eight bits); the slots below it and the
// lowest-index slots at it are gathered and sorted by (energy, slot) in
// shared memory.  Then the controller flags of the population step.
__global__ void __launch_bounds__(kBigThreads)
k_ncm_select_big(int32_t R, int32_t kind, int32_t do_resample, int32_t n_top, int32_t tau,
                 const int64_t *__restrict__ E_src, const int32_t *__restrict__ parent, DevCtl *__restrict__ ctl,
                 int32_t *__restrict__ targets, int32_t *__restrict__ ncm_idx) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ long long red_ll[32];
    __shared__ unsigned int hist[256];
    __shared__ unsigned int s_base[kBigThreads / 32];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned int s_k;
    if (ctl->done) return;
    const int32_t z = ctl->z;
    const bool resampled = z > 1 && do_resample;
    const bool ncm = z > 1 && ctl->enable_cm && ctl->cooldown == 0;
    __syncthreads();
    if (ncm && kind == 0) {
        const int32_t ntop = min(n_top, R);
        long long lmin = LLONG_MAX;
        for (int32_t m = threadIdx.x; m < R; m += blockDim.x) lmin = min(lmin, (long long)E_src[parent[m]]);
        const long long emin = block_reduce(lmin, [](long long a, long long b) { return a < b ? a : b; }, red_ll);
        auto key = [&](int32_t m) { return (unsigned long long)((long long)E_src[parent[m]] - emin); };
        // radix select of the ntop-th smallest key (1-based rank k)
        if (threadIdx.x == 0) { s_prefix = 0ull; s_k = (unsigned)ntop; }
        unsigned long long mask = 0ull;
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
            __syncthreads();
            const unsigned long long pre = s_prefix;
            for (int32_t m = threadIdx.x; m < R; m += blockDim.x) {
                const unsigned long long kk = key(m);
                if ((kk & mask) == pre) atomicAdd(&hist[(kk >> shift) & 0xFFu], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned int k = s_k, b = 0;
                while (hist[b] < k) { k -= hist[b]; ++b; }
                s_k = k;
                s_prefix = pre | ((unsigned long long)b << shift);
            }
            mask |= 0xFFull << shift;
            __syncthreads();
        }
        const unsigned long long kv = s_prefix;   // the ntop-th smallest key
        const unsigned int take_eq = s_k;         // slots at kv to take, lowest indices first
        // gather: keys below kv, and the first take_eq slots (by index) at kv;
        // a contiguous range of slots per thread keeps the index order
        unsigned long long *Ek = reinterpret_cast<unsigned long long *>(sm);
        int32_t P2 = 1;
        while (P2 < ntop) P2 <<= 1;
        int32_t *Mi = reinterpret_cast<int32_t *>(sm + (size_t)P2 * 8);
        const int32_t per = (R + blockDim.x - 1) / blockDim.x;
        const int32_t lo = min(R, (int32_t)threadIdx.x * per), hi = min(R, lo + per);
        unsigned int n_eq = 0, n_lt = 0;
        for (int32_t m = lo; m < hi; ++m) {
            const unsigned long long kk = key(m);
            n_eq += kk == kv ? 1u : 0u;
            n_lt += kk < kv ? 1u : 0u;
        }
        // exclusive prefix over threads of n_eq (for the equal-key quota) and
        // of the number each thread writes
        auto block_excl = [&](unsigned int v) {
            unsigned int x = v;
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            __syncthreads();
            if (lane == 31) s_base[wid] = x;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned int acc = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { const unsigned int c = s_base[w]; s_base[w] = acc; acc += c; }
            }
            __syncthreads();
            return x - v + s_base[wid];
        };
        const unsigned int eq_before = block_excl(n_eq);
        const unsigned int eq_mine = eq_before >= take_eq ? 0u : min(n_eq, take_eq - eq_before);
        const unsigned int out_before = block_excl(n_lt + eq_mine);
        unsigned int o = out_before, eq_taken = 0;
        for (int32_t m = lo; m < hi; ++m) {
            const unsigned long long kk = key(m);
            bool take = kk < kv;
            if (kk == kv && eq_taken < eq_mine) { take = true; ++eq_taken; }
            if (take) { Ek[o] = kk; Mi[o] = m; ++o; }
        }
        for (int32_t x = ntop + threadIdx.x; x < P2; x += blockDim.x) { Ek[x] = ~0ull; Mi[x] = INT32_MAX; }
        __syncthreads();
        for (int32_t k = 2; k <= P2; k <<= 1) {
            for (int32_t j = k >> 1; j > 0; j >>= 1) {
                for (int32_t i = threadIdx.x; i < P2; i += blockDim.x) {
                    const int32_t l = i ^ j;
                    if (l > i) {
                        const unsigned long long ei = Ek[i], el = Ek[l];
                        const int32_t mi = Mi[i], ml = Mi[l];
                        const bool gt = ei > el || (ei == el && mi > ml);
                        if (gt == ((i & k) == 0)) {
                            Ek[i] = el; Ek[l] = ei;
                            Mi[i] = ml; Mi[l] = mi;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int32_t q = threadIdx.x; q < ntop; q += blockDim.x) {
            const int32_t m = Mi[q];
            targets[q] = m;
            ncm_idx[m] = q;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->resampled = resampled ? 1 : 0;
        ctl->ncm_active = ncm ? 1 : 0;
        ctl->ncm_last = ncm ? 1 : 0;
        if (ncm) { ctl->enable_cm = 0; ctl->cooldown = tau; }
    }
}

// ---------------------------------------------------------------- NCM
constexpr int kNcmThreads = 512;

__device__ __forceinline__ bool nbefore(uint32_t ka, int32_t a, uint32_t kb, int32_t b) {
    return ka < kb || (ka == kb && a < b);
}

// One randomised greedy MIS over the iso-sites (stat 0 = candidate,
// 3 = not a candidate).  Decided in rounds: a candidate is taken (1) once
// every coupled candidate earlier in the trial's random order is rejected,
// and rejected (2) once one of them is taken -- the same set the sequential
// greedy scan in that order builds.  Returns the size of the set.
// The rounds are bounded by lim (n + 1 always suffices: every round decides
// at least the earliest undecided candidate); a trial still undecided after
// lim rounds sets PAMC_ERR_TIMEOUT and keeps the set taken so far, which is
// independent, so the move still preserves the energy.
__device__ int32_t mis_trial(int32_t n, const int32_t *rp, const uint32_t *adj, uint8_t *stat,
                             uint32_t *key, int32_t a, int32_t t, int32_t m, uint32_t key0,
                             uint32_t key1, DevCtl *ctl, int *s_flag, int *s_red, int32_t lim) {
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        if (stat[k] != 3) {
            stat[k] = 0;
            key[k] = philox((uint32_t)k, (uint32_t)a, (uint32_t)t, (kTagNcm << 24) | (uint32_t)m, key0, key1).x;
        }
    }
    __syncthreads();
    for (int32_t round = 0; round <= lim; ++round) {
        if (threadIdx.x == 0) *s_flag = 0;
        __syncthreads();
        for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
            if (stat[k] != 0) continue;
            const uint32_t kk = key[k];
            bool any_in = false, all_out = true;
            for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
                const uint32_t w = adj[e];
                if ((w >> 24) == 0) continue;   // zero coupling
                const int32_t j = (int32_t)(w & 0xFFFFFFu);
                const uint8_t sj = *(volatile uint8_t *)&stat[j];
                if (sj == 3 || !nbefore(key[j], j, kk, k)) continue;
                if (sj == 1) any_in = true;
                else if (sj == 0) all_out = false;
            }
            if (any_in) stat[k] = 2;
            else if (all_out) stat[k] = 1;
            else *s_flag = 1;
        }
        __syncthreads();
        const int more = *s_flag;
        __syncthreads();
        if (!more) break;
        if (round == lim && threadIdx.x == 0) atomicExch(&ctl->err, (int)PAMC_ERR_TIMEOUT);
    }
    int32_t c = 0;
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) c += stat[k] == 1 ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (threadIdx.x == 0) *s_red = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicAdd(s_red, c);
    __syncthreads();
    const int32_t tot = *s_red;
    __syncthreads();
    return tot;
}

__host__ __device__ constexpr size_t ncm_stat_bytes(int32_t n) { return ((size_t)n + 15) & ~(size_t)15; }
constexpr size_t kNcmKeySmemMax = 160 * 1024;   // keys join the states in shared memory up to this total

// The cluster move of target q (one CTA), shared by the single-instance and
// the batched kernels.
__device__ __forceinline__ void
ncm_body(int32_t q, int32_t n, const int32_t *__restrict__ rp, const uint32_t *__restrict__ adj, int32_t R,
         int32_t kind, int32_t n_top, int32_t trials, uint32_t key0, uint32_t key1,
         const int8_t *__restrict__ src, const int64_t *__restrict__ E_src,
         const int32_t *__restrict__ parent, const int32_t *__restrict__ targets,
         int8_t *__restrict__ ncm_buf, uint32_t *__restrict__ nkey, int32_t key_smem, int32_t max_rounds,
         DevCtl *__restrict__ ctl, int32_t base, int32_t count, const int32_t *__restrict__ prow) {
    // the per-site decision state of the MIS rounds lives in shared memory
    // (n bytes), and the trial's order keys too (4n bytes) when key_smem:
    // every round reads the state and key of every neighbour
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_flag, s_red;
    __shared__ long long s_e[32];
    if (ctl->done || !ctl->ncm_active || kind != 0) return;
    if (q >= min(n_top, R)) return;
    const int32_t t = ctl->t;
    const int32_t m = targets[q];
    // a population split over processes: this handle moves only its own
    // slots [base, base + count), whose parents sit at rows prow[m - base]
    // of its source buffer (own replicas and the ones it received)
    if (m < base || m - base >= count) return;
    const int8_t *row = src + (size_t)(prow ? prow[m - base] : parent[m]) * n;
    int8_t *sp = ncm_buf + (size_t)q * n;
    uint32_t *key = key_smem ? reinterpret_cast<uint32_t *>(sm + ncm_stat_bytes(n)) : nkey + (size_t)q * n;
    uint8_t *stat = sm;
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) sp[k] = row[k];
    __syncthreads();
    // iso-sites: h_k = 0, so flipping k alone leaves the energy unchanged
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        int32_t h = 0;
        for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
            const uint32_t w = adj[e];
            h += ((int32_t)w >> 24) * sp[w & 0xFFFFFFu];
        }
        stat[k] = h == 0 ? 0 : 3;
    }
    __syncthreads();
    const int32_t lim = max_rounds >= 0 && max_rounds < n + 1 ? max_rounds : n + 1;
    int32_t best = -1, besta = 0;
    for (int32_t a = 0; a < trials; ++a) {
        const int32_t sz = mis_trial(n, rp, adj, stat, key, a, t, m, key0, key1, ctl, &s_flag, &s_red, lim);
        if (sz > best) { best = sz; besta = a; }   // ties keep the earliest trial
    }
    if (trials <= 0) best = 0;
    if (best > 0) {
        mis_trial(n, rp, adj, stat, key, besta, t, m, key0, key1, ctl, &s_flag, &s_red, lim);
        for (int32_t k = threadIdx.x; k < n; k += blockDim.x)
            if (stat[k] == 1) sp[k] = (int8_t)-sp[k];
    }
    __syncthreads();
    // energy check: the move must not change E = -1/2 sum_k s_k h_k
    long long acc = 0;
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        long long h = 0;
        for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
            const uint32_t w = adj[e];
            h += (long long)((int32_t)w >> 24) * sp[w & 0xFFFFFFu];
        }
        acc += (long long)sp[k] * h;
    }
    const long long tot = block_reduce(acc, [](long long x, long long y) { return x + y; }, s_e);
    if (threadIdx.x == 0) {
        long long d = -(tot / 2) - (long long)E_src[parent[m]];
        if (d < 0) d = -d;
        atomicMax((unsigned long long *)&ctl->ncm_dE_max, (unsigned long long)d);
        atomicAdd((unsigned long long *)&ctl->ncm_flipped, (unsigned long long)(best > 0 ? best : 0));
    }
}

__global__ void __launch_bounds__(kNcmThreads)
k_ncm(int32_t n, const int32_t *__restrict__ rp, const uint32_t *__restrict__ adj, int32_t R,
      int32_t kind, int32_t n_top, int32_t trials, uint32_t key0, uint32_t key1,
      const int8_t *__restrict__ src, const int64_t *__restrict__ E_src,
      const int32_t *__restrict__ parent, const int32_t *__restrict__ targets,
      int8_t *__restrict__ ncm_buf, uint32_t *__restrict__ nkey, int32_t key_smem, int32_t max_rounds,
      DevCtl *__restrict__ ctl, int32_t base, int32_t count, const int32_t *__restrict__ prow) {
    ncm_body(blockIdx.x, n, rp, adj, R, kind, n_top, trials, key0, key1, src, E_src, parent, targets, ncm_buf, nkey,
             key_smem, max_rounds, ctl, base, count, prow);
}

// Cluster moves of many instances in one launch: CTA b moves target
// items[b].y of member items[b].x, reading the member's step from its
// controller (the population of step t is sp[t & 1]).
__global__ void __launch_bounds__(kNcmThreads)
k_ncm_batched(const NcmDesc *__restrict__ descs, const int2 *__restrict__ items, int32_t key_smem,
              int32_t max_rounds) {
    const int2 it = items[blockIdx.x];
    const NcmDesc &d = descs[it.x];
    const int32_t t = d.ctl->t;
    if (t >= d.t_end) return;
    ncm_body(it.y, d.n, d.rp, d.adj, d.R, 0, d.n_top, d.trials, d.key0, d.key1, d.sp[t & 1], d.en[t & 1], d.parent,
             d.targets, d.ncm_buf, d.nkey, key_smem, max_rounds, d.ctl, 0, d.R, nullptr);
}

// A restart's re-draw in a batch (after the controller, which advanced t and
// raised redraw): the initial-population draw of step ctl->t for every group
// of four replicas (items (member, chunk of groups)), the energies from the
// definition (items (member, replica)), then the flag is lowered.
__global__ void __launch_bounds__(256)
k_redraw_spins_batched(const RedrawDesc *__restrict__ descs, const int2 *__restrict__ items) {
    const int2 it = items[blockIdx.x];
    const RedrawDesc &d = descs[it.x];
    const DevCtl *ctl = d.ctl;
    if (!ctl->redraw) return;
    const int32_t t = ctl->t, n = d.n, R = d.R;
    int8_t *spins = d.sp[t & 1];
    const int32_t groups = (R + 3) / 4;
    const size_t total = (size_t)groups * n;
    const size_t chunk = (size_t)256 * kRedrawPerThread;
    const size_t lo = (size_t)it.y * chunk, hi = lo + chunk < total ? lo + chunk : total;
    for (size_t x = lo + threadIdx.x; x < hi; x += blockDim.x) {
        const int32_t g = (int32_t)(x / n), i = (int32_t)(x % n);
        const u32x4 u = philox((uint32_t)i, 0u, (uint32_t)t, (kTagInit << 24) | (uint32_t)g, d.key0, d.key1);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int32_t r = 4 * g + q;
            if (r >= R) break;
            int8_t v;
            if (d.kind == 0) v = (w[q] >> 31) ? 1 : -1;
            else v = (int8_t)(((uint64_t)w[q] * (uint64_t)d.K) >> 32);
            spins[(size_t)r * n + i] = v;
        }
    }
}

__global__ void __launch_bounds__(256)
k_redraw_energy_batched(const RedrawDesc *__restrict__ descs, const int2 *__restrict__ items) {
    __shared__ long long red[32];
    const int2 it = items[blockIdx.x];
    const RedrawDesc &d = descs[it.x];
    const DevCtl *ctl = d.ctl;
    if (!ctl->redraw) return;
    const int32_t t = ctl->t, n = d.n, r = it.y;
    const int8_t *s = d.sp[t & 1] + (size_t)r * n;
    long long acc = 0;
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        long long h = 0;
        const int8_t sk = s[k];
        for (int32_t e = d.rp[k]; e < d.rp[k + 1]; ++e) {
            const uint32_t a = d.adj[e];
            const int32_t J = (int32_t)a >> 24;
            if (d.kind == 0) h += (long long)J * s[a & 0xFFFFFFu];
            else h += (s[a & 0xFFFFFFu] == sk) ? J : 0;
        }
        acc += d.kind == 0 ? (long long)sk * h : h;
    }
    const long long tot = block_reduce(acc, [](long long x, long long y) { return x + y; }, red);
    if (threadIdx.x == 0) d.en[t & 1][r] = d.kind == 0 ? -(tot / 2) : (-tot - d.Wsum);
}

__global__ void k_redraw_done_batched(const RedrawDesc *__restrict__ descs, int32_t nmem) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nmem) descs[i].ctl->redraw = 0;
}

// ---------------------------------------------------------------- controller
constexpr int kCtlThreads = 1024;

// Entry i of the last w history values counts as distinct when no earlier
// entry of that window holds the same value; one entry per thread, summed by
// the barrier count (the history sits in shared memory).
__device__ __forceinline__ bool distinct_entry(const long long *h, int32_t len, int32_t w, int32_t i) {
    if (w > len) w = len;
    if (i < len - w || i >= len) return false;
    for (int32_t q = len - w; q < i; ++q)
        if (h[q] == h[i]) return false;
    return true;
}

__device__ __forceinline__ void
control_body(int32_t n, int64_t W, int32_t R, int32_t stagnation, int32_t z_rst, int32_t win_short,
             int32_t win_long, int32_t max_ds, int32_t max_dl, double reheat, double beta0,
             int64_t target, const int64_t *__restrict__ E, const int8_t *__restrict__ spins,
             int8_t *__restrict__ best, DevCtl *__restrict__ ctl, int32_t base, int32_t count) {
    // E holds all R energies; spins only rows [base, base + count) of the
    // population (all of it unless the population is split over processes)
    __shared__ long long s_e[32];
    __shared__ int s_i[32];
    __shared__ int s_improved, s_rb;
    __shared__ long long s_hist[kHistMax];
    __shared__ int s_len, s_gate;
    if (ctl->done) return;
    // argmin of (E, index): the replica with the largest cut, lowest index on ties
    long long be = LLONG_MAX;
    int bi = 0x7fffffff;
    for (int32_t r = threadIdx.x; r < R; r += blockDim.x) {
        const long long e = E[r];
        if (e < be || (e == be && r < bi)) { be = e; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long e2 = __shfl_down_sync(0xffffffffu, be, o);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        if (e2 < be || (e2 == be && i2 < bi)) { be = e2; bi = i2; }
    }
    if ((threadIdx.x & 31) == 0) { s_e[threadIdx.x >> 5] = be; s_i[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (s_e[w] < be || (s_e[w] == be && s_i[w] < bi)) { be = s_e[w]; bi = s_i[w]; }
        const long long cut = (W - be) / 2;
        s_improved = cut > ctl->mstar;
        s_rb = bi;
        if (s_improved) {
            ctl->mstar = cut;
            ctl->best_replica = bi;
            ctl->best_owned = bi >= base && bi - base < count ? 1 : 0;
        }
    }
    __syncthreads();
    if (s_improved && s_rb >= base && s_rb - base < count) {
        const int8_t *row = spins + (size_t)(s_rb - base) * n;
        for (int32_t k = threadIdx.x; k < n; k += blockDim.x) best[k] = row[k];
    }
    DevCtl &c = *ctl;
    // record M* in the recent-progress history (the last max(windows) values),
    // shifted in shared memory and written back by all threads
    const int32_t len0 = c.hist_len;
    for (int32_t i = threadIdx.x; i < len0; i += blockDim.x) s_hist[i] = c.hist[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t hl = win_long > win_short ? win_long : win_short;
        if (hl > kHistMax) hl = kHistMax;
        int32_t len = len0;
        if (hl > 0) {
            if (len == hl) {
                for (int32_t i = 0; i + 1 < hl; ++i) s_hist[i] = s_hist[i + 1];
                len = hl - 1;
            }
            s_hist[len++] = c.mstar;
        }
        s_len = len;
        s_gate = stagnation && c.cooldown == 0 && hl > 0 && len >= hl;
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < s_len; i += blockDim.x) c.hist[i] = s_hist[i];
    if (threadIdx.x == 0) c.hist_len = s_len;
    int32_t ds = 0, dl = 0;
    if (s_gate) {   // uniform over the block
        ds = __syncthreads_count(distinct_entry(s_hist, s_len, win_short, (int32_t)threadIdx.x));
        dl = __syncthreads_count(distinct_entry(s_hist, s_len, win_long, (int32_t)threadIdx.x));
    }
    if (threadIdx.x != 0) return;
    if (s_gate) {
        if (ds <= max_ds && dl <= max_dl) {
            c.beta = __dmul_rn(reheat, c.beta);
            c.delta = c.dbeta;
            c.enable_cm = 1;
        } else if (ds <= max_ds) {
            if (c.beta > beta0) c.delta = -c.dbeta;
        } else {
            c.delta = c.dbeta;
        }
    }
    c.restart = 0;
    if (z_rst > 0 && c.z >= z_rst) {
        c.cycle += 1;
        c.z = 1;
        c.beta = beta0;
        c.delta = c.dbeta;
        c.enable_cm = 0;
        c.cooldown = 0;
        c.hist_len = 0;
        c.restart = 1;
        c.redraw = 1;   // consumed by a batch's re-draw (a single run re-draws by step index)
    } else {
        c.z += 1;
        c.beta = __dadd_rn(c.beta, c.delta);
        if (c.cooldown > 0) c.cooldown -= 1;
    }
    c.t += 1;
    if (target >= 0 && c.mstar >= target) c.done = 1;
}

__global__ void __launch_bounds__(kCtlThreads)
k_control(int32_t n, int64_t W, int32_t R, int32_t stagnation, int32_t z_rst, int32_t win_short,
          int32_t win_long, int32_t max_ds, int32_t max_dl, double reheat, double beta0,
          int64_t target, const int64_t *__restrict__ E, const int8_t *__restrict__ spins,
          int8_t *__restrict__ best, DevCtl *__restrict__ ctl, int32_t base, int32_t count) {
    control_body(n, W, R, stagnation, z_rst, win_short, win_long, max_ds, max_dl, reheat, beta0, target, E,
                 spins, best, ctl, base, count);
}

__global__ void __launch_bounds__(kCtlThreads) k_control_batched(const CtlDesc *__restrict__ descs) {
    const CtlDesc d = descs[blockIdx.x];
    // every thread reads t before control_body's first barrier; thread 0 advances it afterwards
    const int32_t t = d.ctl->t;
    if (t >= d.t_end) return;
    control_body(d.n, d.W, d.R, d.stagnation, d.z_rst, d.win_short, d.win_long, d.max_ds, d.max_dl,
                 d.reheat, d.beta0, d.target, d.en[(t + 1) & 1], d.sp[(t + 1) & 1], d.best, d.ctl, 0, d.R);
}

}  // namespace

cudaError_t launch_tables(int kind, int rule, int32_t H, const DevCtl *ctl, uint64_t *tab,
                          cudaStream_t st) {
    if (kind == 1 && rule == 2) {
        k_tables_softmax<<<1, 256, 0, st>>>(H, ctl, reinterpret_cast<float *>(tab));
    } else if (kind == 0) {
        int grid = (2 * H + 1 + 255) / 256;   // wide field ranges: many entries
        if (grid > 304) grid = 304;
        k_tables<<<grid, 256, 0, st>>>(kind, rule, H, ctl, tab);
    } else {
        const int32_t W1 = 4 * H + 1;
        int grid = (W1 * W1 + W1 + 255) / 256;
        if (grid > 304) grid = 304;
        k_tables<<<grid, 256, (size_t)W1 * sizeof(double), st>>>(kind, rule, H, ctl, tab);
    }
    return cudaGetLastError();
}

// R prefix sums (8 bytes) and R counts (4 bytes), sized for the next power of
// two of R so that the NCM target sort can pad to it
size_t prep_smem_bytes(int32_t R) {
    size_t P2 = 1;
    while (P2 < (size_t)(R > 1 ? R : 1)) P2 <<= 1;
    return P2 * 8 + P2 * 4;
}

size_t ncm_select_smem_bytes(int32_t n_top) {
    size_t P2 = 1;
    while (P2 < (size_t)(n_top > 1 ? n_top : 1)) P2 <<= 1;
    return P2 * 8 + P2 * 4;
}

cudaError_t launch_prep(const pamc_params &p, const int64_t *E_src, DevCtl *ctl, int32_t *parent,
                        int32_t *count, int32_t *ncm_idx, int32_t *targets, int32_t *fam, uint64_t *qbuf,
                        cudaStream_t st, long long *mm) {
    if (p.R > kPrepOneCtaMaxR) {
        if (!qbuf || !mm) return cudaErrorInvalidValue;
        const int fam_reset = p.z_rst > 0 && p.restart_reinit ? 1 : 0;
        const int32_t ntop = p.n_top < p.R ? p.n_top : p.R;
        const size_t sel_smem = ncm_select_smem_bytes(ntop);
        cudaError_t err = allow_dynamic_smem(k_ncm_select_big, sel_smem);
        if (err != cudaSuccess) return err;
        k_minmax<<<1, kBigThreads, 0, st>>>(p.R, p.resample, E_src, ctl, mm);
        k_weights<<<(p.R + kWeightThreads - 1) / kWeightThreads, kWeightThreads, 0, st>>>(p.R, p.kind, p.resample,
                                                                                          E_src, ctl, qbuf, mm);
        k_scan_big<<<1, kBigThreads, 0, st>>>(p.R, p.resample, qbuf, ctl);
        err = cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)p.R, st);
        if (err != cudaSuccess) return err;
        k_parent_big<<<(p.R + 255) / 256, 256, 0, st>>>(p.R, p.resample, (uint32_t)p.seed, (uint32_t)(p.seed >> 32),
                                                        qbuf, ctl, parent, count, ncm_idx, fam, fam_reset);
        k_ncm_select_big<<<1, kBigThreads, sel_smem, st>>>(p.R, p.kind, p.resample, p.n_top, p.cooldown_tau, E_src,
                                                           parent, ctl, targets, ncm_idx);
        return cudaGetLastError();
    }
    const size_t smem = prep_smem_bytes(p.R);
    cudaError_t err = allow_dynamic_smem(k_prep, smem);
    if (err != cudaSuccess) return err;
    if (qbuf)
        k_weights<<<(p.R + kWeightThreads - 1) / kWeightThreads, kWeightThreads, 0, st>>>(p.R, p.kind, p.resample,
                                                                                          E_src, ctl, qbuf, nullptr);
    k_prep<<<1, kPrepThreads, smem, st>>>(p.R, p.kind, p.resample, p.n_top, p.cooldown_tau,
                                          (uint32_t)p.seed, (uint32_t)(p.seed >> 32), E_src, ctl,
                                          parent, count, ncm_idx, targets, fam,
                                          p.z_rst > 0 && p.restart_reinit ? 1 : 0, qbuf);
    return cudaGetLastError();
}

cudaError_t launch_ncm(int32_t n, const int32_t *rp, const uint32_t *adj, const pamc_params &p,
                       const int8_t *src, const int64_t *E_src, const int32_t *parent,
                       const int32_t *targets, int8_t *ncm_buf, uint32_t *nkey, DevCtl *ctl,
                       cudaStream_t st, int32_t base, int32_t count, const int32_t *prow) {
    const int32_t ntop = p.n_top < p.R ? p.n_top : p.R;
    if (ntop <= 0 || p.kind != 0 || !p.stagnation) return cudaSuccess;
    const size_t with_keys = ncm_stat_bytes(n) + (size_t)n * 4;
    const int key_smem = with_keys <= kNcmKeySmemMax ? 1 : 0;
    const size_t smem = key_smem ? with_keys : ncm_stat_bytes(n);
    cudaError_t err = allow_dynamic_smem(k_ncm, smem);
    if (err != cudaSuccess) return err;
    // PAMC_NCM_MAX_ROUNDS: a smaller bound on the MIS rounds than n + 1, for
    // tests that make the bounded wait run out (PAMC_ERR_TIMEOUT, pamc_sync)
    int32_t max_rounds = -1;
    if (const char *env = getenv("PAMC_NCM_MAX_ROUNDS")) max_rounds = atoi(env);
    k_ncm<<<ntop, kNcmThreads, smem, st>>>(n, rp, adj, p.R, p.kind, p.n_top, p.mis_trials,
                                           (uint32_t)p.seed, (uint32_t)(p.seed >> 32), src, E_src,
                                           parent, targets, ncm_buf, nkey, key_smem, max_rounds, ctl, base,
                                           count < 0 ? p.R : count, prow);
    return cudaGetLastError();
}

cudaError_t launch_control(int32_t n, int64_t W, const pamc_params &p, const int64_t *E,
                           const int8_t *spins, int8_t *best, DevCtl *ctl, cudaStream_t st, int32_t base,
                           int32_t count) {
    k_control<<<1, kCtlThreads, 0, st>>>(n, W, p.R, p.stagnation, p.z_rst, p.win_short, p.win_long,
                                         p.max_distinct_short, p.max_distinct_long, p.reheat_factor,
                                         p.beta0, p.target_cut, E, spins, best, ctl, base,
                                         count < 0 ? p.R : count);
    return cudaGetLastError();
}

cudaError_t launch_population_batched(const PrepDesc *prep, const TabDesc *tabs, int32_t ninst,
                                      int32_t R_max, cudaStream_t st) {
    if (ninst <= 0) return cudaSuccess;
    const size_t smem = prep_smem_bytes(R_max);
    cudaError_t err = allow_dynamic_smem(k_prep_batched, smem);
    if (err != cudaSuccess) return err;
    k_prep_batched<<<ninst, kPrepThreads, smem, st>>>(prep);
    k_tables_batched<<<ninst * kTabBlocks, 256, 0, st>>>(tabs);
    return cudaGetLastError();
}

cudaError_t launch_ncm_batched(const NcmDesc *descs, const int2 *items, int32_t nitems, int32_t n_max,
                               cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const size_t with_keys = ncm_stat_bytes(n_max) + (size_t)n_max * 4;
    const int key_smem = with_keys <= kNcmKeySmemMax ? 1 : 0;
    const size_t smem = key_smem ? with_keys : ncm_stat_bytes(n_max);
    cudaError_t err = allow_dynamic_smem(k_ncm_batched, smem);
    if (err != cudaSuccess) return err;
    int32_t max_rounds = -1;
    if (const char *env = getenv("PAMC_NCM_MAX_ROUNDS")) max_rounds = atoi(env);
    k_ncm_batched<<<nitems, kNcmThreads, smem, st>>>(descs, items, key_smem, max_rounds);
    return cudaGetLastError();
}

cudaError_t launch_redraw_batched(const RedrawDesc *descs, int32_t nmem, const int2 *spin_items, int32_t nspin,
                                  const int2 *energy_items, int32_t nenergy, cudaStream_t st) {
    if (nmem <= 0) return cudaSuccess;
    if (nspin > 0) k_redraw_spins_batched<<<nspin, 256, 0, st>>>(descs, spin_items);
    if (nenergy > 0) k_redraw_energy_batched<<<nenergy, 256, 0, st>>>(descs, energy_items);
    k_redraw_done_batched<<<(nmem + 127) / 128, 128, 0, st>>>(descs, nmem);
    return cudaGetLastError();
}

cudaError_t launch_control_batched(const CtlDesc *descs, int32_t ninst, cudaStream_t st) {
    if (ninst <= 0) return cudaSuccess;
    k_control_batched<<<ninst, kCtlThreads, 0, st>>>(descs);
    return cudaGetLastError();
}

}  // namespace pamc
