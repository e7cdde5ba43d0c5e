// sweep.cu -- S single-spin sweeps per temperature step over the whole
// population (Algorithm 1, "Run S MCMC updates on every replica at beta"),
// plus the random (re)initialisation of the population.
//
// Ising (Eq. 3-4): for vertex k with field h_k = sum_j J_kj s_j, heat-bath
// sets s_k = +1 iff u < T(h_k); Metropolis flips iff u < T_M(2 s_k h_k).
// Potts K=3 (Eq. 6-7, Suppl. S3): with syn_c(k) = sum_j J_kj [sigma_j = c],
// label 0 iff u0 < T1(syn1-syn0, syn2-syn0), else label 1 iff
// u1 < T2(syn2-syn1), else label 2.
//
// GB300 layout.  One replica GROUP shares one Philox call per vertex visit:
// 4 Ising replicas (the four 32-bit words) or 2 Potts replicas (two words
// each).  A group's spins live in shared memory as one byte per vertex
// (Ising: one bit per replica; Potts: two bits per replica), so a torus
// replica of 19,881 spins costs 19.9 KB for four replicas.  Fields are not
// stored: each visit pulls them from the neighbours' packed spins with
// byte-lane SIMD (every neighbour adds its 0/1 bits, spread into bytes, to a
// positive- or negative-coupling accumulator), so no atomics and no field
// arrays are needed and the result is the exact integer field.  Several warps
// cooperate on one group: each level of the (t, sweep) schedule is a set of
// pairwise-uncoupled vertices, processed in parallel, with a named barrier
// between levels; several groups share a CTA.  The end-of-step energy is
// recomputed from the definition, E = -1/2 sum_k s_k h_k (Ising) or
// E = -sum_k syn_{sigma_k}(k) - W (Potts), which is the full-recompute check
// of the incrementally updated state.
#include "pamc_device.cuh"
#include "pamc_internal.h"

namespace pamc {

namespace {

__device__ __forceinline__ void group_barrier(int id, int nthreads, int groups) {
    if (groups == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
}

// source row of slot r: the NCM buffer if the cluster move rewrote it, else
// the resampling parent in the previous population
__device__ __forceinline__ const int8_t *src_row(int32_t r, int32_t n, const int8_t *src,
                                                 const int32_t *parent, const int8_t *ncm_buf,
                                                 const int32_t *ncm_idx) {
    const int32_t q = ncm_idx[r];
    if (q >= 0) return ncm_buf + (size_t)q * n;
    return src + (size_t)parent[r] * n;
}

template <int KIND, bool ELLP>
__global__ void __launch_bounds__(1024)
k_sweep(int32_t n, int32_t n_pad, const int32_t *__restrict__ rp, const uint32_t *__restrict__ adj,
        int32_t H, int32_t R, int32_t S, int32_t rule, uint32_t key0, uint32_t key1, int32_t t,
        int32_t slot, const int32_t *__restrict__ sorder, const int32_t *__restrict__ slvl,
        const int32_t *__restrict__ snlev, const uint32_t *__restrict__ sell, int32_t W,
        const uint64_t *__restrict__ tab,
        const int8_t *__restrict__ src, const int32_t *__restrict__ parent,
        const int8_t *__restrict__ ncm_buf, const int32_t *__restrict__ ncm_idx,
        int8_t *__restrict__ dst, int64_t *__restrict__ E_dst, const DevCtl *__restrict__ ctl,
        int64_t Wsum, int gpc, int tpg) {
    constexpr int RPG = KIND == 0 ? 4 : 2;   // replicas per Philox call
    extern __shared__ __align__(16) uint8_t smem[];
    if (ctl->done) return;

    // shared layout: [table][group spins][energy partials]
    const int tabn = KIND == 0 ? (2 * H + 1) : (4 * H + 1);
    uint64_t *tab_s = reinterpret_cast<uint64_t *>(smem);
    uint8_t *spins_all = smem + (size_t)tabn * 8;
    unsigned long long *red = reinterpret_cast<unsigned long long *>(
        spins_all + (size_t)gpc * n_pad);
    for (int i = threadIdx.x; i < tabn; i += blockDim.x)
        tab_s[i] = tab[(KIND == 0 ? 0 : (size_t)(4 * H + 1) * (4 * H + 1)) + i];
    for (int i = threadIdx.x; i < gpc * RPG; i += blockDim.x) red[i] = 0ull;

    const int gl = threadIdx.x / tpg, li = threadIdx.x % tpg;
    const int32_t g = blockIdx.x * gpc + gl;
    const int32_t r0 = g * RPG;
    const bool active = r0 < R;
    uint8_t *sp = spins_all + (size_t)gl * n_pad;

    if (active) {
        const int8_t *rows[RPG];
#pragma unroll
        for (int q = 0; q < RPG; ++q)
            rows[q] = (r0 + q < R) ? src_row(r0 + q, n, src, parent, ncm_buf, ncm_idx) : nullptr;
        for (int32_t k = li; k < n; k += tpg) {
            uint32_t b = 0;
#pragma unroll
            for (int q = 0; q < RPG; ++q) {
                if (rows[q] == nullptr) continue;
                const int8_t v = rows[q][k];
                if (KIND == 0) b |= (uint32_t)(v > 0) << q;
                else b |= (uint32_t)(v & 3) << (2 * q);
            }
            sp[k] = (uint8_t)b;
        }
    }
    __syncthreads();

    const uint64_t *T1 = tab;   // Potts: (4H+1)^2 table in global memory
    const int W1 = 4 * H + 1;

    if (active) {
        const size_t ell_stride = (size_t)(((n + 31) >> 5) << 5) * W;
        for (int32_t sw = 0; sw < S; ++sw) {
            const size_t sb = (size_t)slot * S + sw;
            const int32_t *ord = sorder + sb * (size_t)n;
            const int32_t *lp = slvl + sb * (size_t)(n + 1);
            const uint32_t *es = ELLP ? sell + sb * ell_stride : nullptr;
            const int32_t L = snlev[sb];
            for (int32_t lev = 0; lev < L; ++lev) {
                const int32_t beg = lp[lev], end = lp[lev + 1];
                for (int32_t i = beg + li; i < end; i += tpg) {
                    const uint32_t a0 = (uint32_t)ord[i];
                    const int32_t k = (int32_t)(a0 & 0xFFFFFFu);
                    // neighbour words: position-indexed ELL (coalesced, no
                    // dependence on k) or the CSR row of k
                    const uint32_t *ep;
                    int32_t cnt, stride;
                    if (ELLP) {
                        ep = es + (size_t)(i >> 5) * 32 * W + (i & 31);
                        cnt = (int32_t)(a0 >> 24);
                        stride = 32;
                    } else {
                        const int32_t e0 = rp[k];
                        ep = adj + e0;
                        cnt = rp[k + 1] - e0;
                        stride = 1;
                    }
                    const u32x4 u = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t,
                                           (kTagFlip << 24) | (uint32_t)g, key0, key1);
                    const uint32_t oldb = sp[k];
                    uint32_t newb = 0;
                    if (KIND == 0) {
                        uint32_t accP = 0, accN = 0;
                        int32_t jsum = 0;
#pragma unroll 4
                        for (int32_t s2 = 0; s2 < cnt; ++s2) {
                            const uint32_t a = ep[(size_t)s2 * stride];
                            const int32_t j = (int32_t)(a & 0xFFFFFFu);
                            const int32_t J = (int32_t)a >> 24;
                            const uint32_t x = ((uint32_t)sp[j] * 0x00204081u) & 0x01010101u;
                            if (J > 0) accP += x * (uint32_t)J;
                            else accN += x * (uint32_t)(-J);
                            jsum += J;
                        }
                        const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int32_t P = (int32_t)((accP >> (8 * q)) & 0xFFu);
                            const int32_t N = (int32_t)((accN >> (8 * q)) & 0xFFu);
                            const int32_t h = 2 * (P - N) - jsum;
                            const uint32_t s = (oldb >> q) & 1u;
                            uint32_t ns;
                            if (rule == 0) {
                                ns = ((uint64_t)uw[q] < tab_s[h + H]) ? 1u : 0u;
                            } else {
                                const int32_t sh = s ? h : -h;
                                ns = ((uint64_t)uw[q] < tab_s[sh + H]) ? (s ^ 1u) : s;
                            }
                            newb |= ns << q;
                        }
                    } else {
                        uint32_t P0 = 0, N0 = 0, P1 = 0, N1 = 0;
#pragma unroll 4
                        for (int32_t s2 = 0; s2 < cnt; ++s2) {
                            const uint32_t a = ep[(size_t)s2 * stride];
                            const int32_t j = (int32_t)(a & 0xFFFFFFu);
                            const int32_t J = (int32_t)a >> 24;
                            const uint32_t nb = sp[j];
                            const uint32_t x0 = 1u << (8 * (nb & 3u));
                            const uint32_t x1 = 1u << (8 * ((nb >> 2) & 3u));
                            if (J > 0) { P0 += x0 * (uint32_t)J; P1 += x1 * (uint32_t)J; }
                            else { N0 += x0 * (uint32_t)(-J); N1 += x1 * (uint32_t)(-J); }
                        }
                        const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const uint32_t Pq = q ? P1 : P0, Nq = q ? N1 : N0;
                            const int32_t s0 = (int32_t)(Pq & 0xFFu) - (int32_t)(Nq & 0xFFu);
                            const int32_t s1 = (int32_t)((Pq >> 8) & 0xFFu) - (int32_t)((Nq >> 8) & 0xFFu);
                            const int32_t s2 = (int32_t)((Pq >> 16) & 0xFFu) - (int32_t)((Nq >> 16) & 0xFFu);
                            const int32_t a1 = s1 - s0, b1 = s2 - s0, c2 = s2 - s1;
                            const uint64_t t1 = __ldg(&T1[(size_t)(a1 + 2 * H) * W1 + (b1 + 2 * H)]);
                            uint32_t lab;
                            if ((uint64_t)uw[2 * q] < t1) lab = 0;
                            else if ((uint64_t)uw[2 * q + 1] < tab_s[c2 + 2 * H]) lab = 1;
                            else lab = 2;
                            newb |= lab << (2 * q);
                        }
                    }
                    if (newb != oldb) sp[k] = (uint8_t)newb;
                }
                group_barrier(1 + gl, tpg, gpc);
            }
        }

        // energy from the definition, and write-back of the spins
        long long acc[RPG];
#pragma unroll
        for (int q = 0; q < RPG; ++q) acc[q] = 0;
        for (int32_t k = li; k < n; k += tpg) {
            const uint32_t b = sp[k];
            const int32_t e0 = rp[k], e1 = rp[k + 1];
            if (KIND == 0) {
                uint32_t accP = 0, accN = 0;
                int32_t jsum = 0;
                for (int32_t e = e0; e < e1; ++e) {
                    const uint32_t a = adj[e];
                    const int32_t j = (int32_t)(a & 0xFFFFFFu);
                    const int32_t J = (int32_t)a >> 24;
                    const uint32_t x = ((uint32_t)sp[j] * 0x00204081u) & 0x01010101u;
                    if (J > 0) accP += x * (uint32_t)J;
                    else accN += x * (uint32_t)(-J);
                    jsum += J;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int32_t P = (int32_t)((accP >> (8 * q)) & 0xFFu);
                    const int32_t N = (int32_t)((accN >> (8 * q)) & 0xFFu);
                    const int32_t h = 2 * (P - N) - jsum;
                    const int32_t s = ((b >> q) & 1u) ? 1 : -1;
                    acc[q] += (long long)(s * h);
                    if (r0 + q < R) dst[(size_t)(r0 + q) * n + k] = (int8_t)s;
                }
            } else {
                uint32_t P0 = 0, N0 = 0, P1 = 0, N1 = 0;
                for (int32_t e = e0; e < e1; ++e) {
                    const uint32_t a = adj[e];
                    const int32_t j = (int32_t)(a & 0xFFFFFFu);
                    const int32_t J = (int32_t)a >> 24;
                    const uint32_t nb = sp[j];
                    const uint32_t x0 = 1u << (8 * (nb & 3u));
                    const uint32_t x1 = 1u << (8 * ((nb >> 2) & 3u));
                    if (J > 0) { P0 += x0 * (uint32_t)J; P1 += x1 * (uint32_t)J; }
                    else { N0 += x0 * (uint32_t)(-J); N1 += x1 * (uint32_t)(-J); }
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint32_t lab = (b >> (2 * q)) & 3u;
                    const uint32_t Pq = q ? P1 : P0, Nq = q ? N1 : N0;
                    const int32_t syn = (int32_t)((Pq >> (8 * lab)) & 0xFFu) -
                                        (int32_t)((Nq >> (8 * lab)) & 0xFFu);
                    acc[q] += (long long)syn;
                    if (r0 + q < R) dst[(size_t)(r0 + q) * n + k] = (int8_t)lab;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RPG; ++q) {
            long long v = acc[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&red[gl * RPG + q], (unsigned long long)v);
        }
    }
    __syncthreads();
    if (active && li < RPG && r0 + li < R) {
        const long long tot = (long long)red[gl * RPG + li];
        E_dst[r0 + li] = KIND == 0 ? -(tot / 2) : (-tot - Wsum);
    }
}

// Random initial population: Ising s = +1 iff the top bit of the draw is set,
// Potts sigma = floor(3 u / 2^32); draw = Philox(i, 0, t, INIT<<24 | r/4)[r%4].
__global__ void k_init_spins(int kind, int32_t K, int32_t n, int32_t R, uint32_t key0, uint32_t key1,
                             int32_t t, int only_if_restart, const DevCtl *__restrict__ ctl,
                             int8_t *__restrict__ spins) {
    // a restart re-draws the population in the iteration that restarted
    // (the controller has then advanced t to the key t)
    if (only_if_restart && !(ctl->restart && ctl->t == t)) return;
    const int32_t groups = (R + 3) / 4;
    const size_t total = (size_t)groups * n;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
         x += (size_t)gridDim.x * blockDim.x) {
        const int32_t g = (int32_t)(x / n), i = (int32_t)(x % n);
        const u32x4 u = philox((uint32_t)i, 0u, (uint32_t)t, (kTagInit << 24) | (uint32_t)g, key0, key1);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int32_t r = 4 * g + q;
            if (r >= R) break;
            int8_t v;
            if (kind == 0) v = (w[q] >> 31) ? 1 : -1;
            else v = (int8_t)(((uint64_t)w[q] * (uint64_t)K) >> 32);
            spins[(size_t)r * n + i] = v;
        }
    }
}

// Energy of every replica from the definition (one CTA per replica).
__global__ void k_energy(int kind, int32_t n, const int32_t *__restrict__ rp,
                         const uint32_t *__restrict__ adj, int32_t R, int only_if_restart,
                         const DevCtl *__restrict__ ctl, int64_t Wsum, int32_t t,
                         const int8_t *__restrict__ spins, int64_t *__restrict__ E) {
    if (only_if_restart && !(ctl->restart && ctl->t == t)) return;
    __shared__ long long red[32];
    const int32_t r = blockIdx.x;
    const int8_t *s = spins + (size_t)r * n;
    long long acc = 0;
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        long long h = 0;
        const int8_t sk = s[k];
        for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
            const uint32_t a = adj[e];
            const int32_t j = (int32_t)(a & 0xFFFFFFu);
            const int32_t J = (int32_t)a >> 24;
            if (kind == 0) h += (long long)J * s[j];
            else h += (s[j] == sk) ? J : 0;
        }
        acc += kind == 0 ? (long long)sk * h : h;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        E[r] = kind == 0 ? -(tot / 2) : (-tot - Wsum);
    }
}

}  // namespace

size_t sweep_smem_bytes(int kind, int32_t n, int32_t H, SweepCfg cfg) {
    if (kind == 0) return sweep_ising_smem_bytes(n, H, cfg);
    if (kind == 2) return sweep_softmax_smem_bytes(n, H, cfg);
    const int RPG = kind == 0 ? 4 : 2;
    const int tabn = kind == 0 ? (2 * H + 1) : (4 * H + 1);
    const int32_t n_pad = (n + 15) & ~15;
    return (size_t)tabn * 8 + (size_t)cfg.groups_per_cta * n_pad + (size_t)cfg.groups_per_cta * RPG * 8;
}

cudaError_t launch_sweep(int kind, int rule, int32_t n, const int32_t *rp, const uint32_t *adj,
                         int32_t H, const pamc_params &p, int32_t t, int32_t slot, SchedView sv,
                         const uint64_t *tab, const int8_t *src, const int32_t *parent,
                         const int8_t *ncm_buf, const int32_t *ncm_idx, int8_t *dst,
                         int64_t *E_dst, const DevCtl *ctl, SweepCfg cfg, int64_t Wsum,
                         cudaStream_t st) {
    if (kind == 0)
        return launch_sweep_ising(rule, n, rp, adj, H, p, t, slot, sv, tab, src, parent, ncm_buf,
                                  ncm_idx, dst, E_dst, ctl, cfg, st);
    if (kind == 2)
        return launch_sweep_softmax(n, rp, adj, H, p, t, slot, sv, tab, src, parent, ncm_idx, dst, E_dst, ctl,
                                    cfg, Wsum, st);
    const int RPG = kind == 0 ? 4 : 2;
    const int32_t groups = (p.R + RPG - 1) / RPG;
    const int gpc = cfg.groups_per_cta, tpg = cfg.warps_per_group * 32;
    const int32_t n_pad = (n + 15) & ~15;
    const size_t smem = sweep_smem_bytes(kind, n, H, cfg);
    const int grid = (groups + gpc - 1) / gpc;
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    cudaError_t err;
#define PAMC_LAUNCH_SWEEP(KD, EL)                                                                \
    do {                                                                                         \
        err = allow_dynamic_smem(k_sweep<KD, EL>, smem);                                         \
        if (err != cudaSuccess) return err;                                                      \
        k_sweep<KD, EL><<<grid, gpc * tpg, smem, st>>>(                                          \
            n, n_pad, rp, adj, H, p.R, p.sweeps, rule, k0, k1, t, slot, sv.order, sv.lvl_ptr,    \
            sv.nlev, sv.ell, sv.W, tab, src, parent, ncm_buf, ncm_idx, dst, E_dst, ctl, Wsum,    \
            gpc, tpg);                                                                           \
    } while (0)
    const bool ell = sv.ell != nullptr;
    if (ell) PAMC_LAUNCH_SWEEP(1, true);
    else PAMC_LAUNCH_SWEEP(1, false);
#undef PAMC_LAUNCH_SWEEP
    return cudaGetLastError();
}

cudaError_t launch_init(int kind, int32_t K, int32_t n, const int32_t *rp, const uint32_t *adj, int32_t R,
                        uint64_t seed, int32_t t, int only_if_restart, const DevCtl *ctl,
                        int64_t Wsum, int8_t *spins, int64_t *E, cudaStream_t st) {
    const size_t total = (size_t)((R + 3) / 4) * n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_init_spins<<<grid, 256, 0, st>>>(kind, K, n, R, (uint32_t)seed, (uint32_t)(seed >> 32), t,
                                        only_if_restart, ctl, spins);
    k_energy<<<R, 256, 0, st>>>(kind, n, rp, adj, R, only_if_restart, ctl, Wsum, t, spins, E);
    return cudaGetLastError();
}

cudaError_t launch_energy(int kind, int32_t n, const int32_t *rp, const uint32_t *adj, int32_t R,
                          const DevCtl *ctl, int64_t Wsum, const int8_t *spins, int64_t *E, cudaStream_t st) {
    k_energy<<<R, 256, 0, st>>>(kind, n, rp, adj, R, 0, ctl, Wsum, 0, spins, E);
    return cudaGetLastError();
}

cudaError_t launch_init_spins(int kind, int32_t K, int32_t n, int32_t R, uint64_t seed, int32_t t,
                              int only_if_restart, const DevCtl *ctl, int8_t *spins, cudaStream_t st) {
    const size_t total = (size_t)((R + 3) / 4) * n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_init_spins<<<grid, 256, 0, st>>>(kind, K, n, R, (uint32_t)seed, (uint32_t)(seed >> 32), t,
                                        only_if_restart, ctl, spins);
    return cudaGetLastError();
}

}  // namespace pamc
