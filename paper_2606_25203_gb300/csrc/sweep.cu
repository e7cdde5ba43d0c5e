// sweep.cu -- the random (re)initialisation of the population and its
// energies from the definition, and the dispatch of the S sweeps of a
// temperature step (Algorithm 1, "Run S MCMC updates on every replica at
// beta") to the kernel of the model: sweep_ising.cu (Ising, Eq. 3-4),
// sweep_potts.cu (three-state Potts, cascaded sampler of Suppl. S3) and
// sweep_softmax.cu (K-state Potts, softmax noisy argmax of Sec. III.F, Eq. 8-9).
//
// Initial values: replica r's value at vertex i comes from word r mod 4 of
// Philox(i, 0, t, INIT<<24 | r/4), r the replica's index in the whole
// population: s = +1 iff the top bit is set (Ising), or
// label floor(K u / 2^32) (Potts).  Energies: E = -1/2 sum_k s_k h_k (Ising),
// E = -sum_k syn_{sigma_k}(k) - W (Potts).
#include "pamc_device.cuh"
#include "pamc_internal.h"

namespace pamc {

namespace {

__global__ void k_init_spins(int kind, int32_t K, int32_t n, int32_t R, uint32_t key0, uint32_t key1,
                             int32_t t, int only_if_restart, const DevCtl *__restrict__ ctl,
                             int8_t *__restrict__ spins, int32_t gbase) {
    // a restart re-draws the population in the iteration that restarted
    // (the controller has then advanced t to the key t)
    if (only_if_restart && !(ctl->restart && ctl->t == t)) return;
    const int32_t groups = (R + 3) / 4;
    const size_t total = (size_t)groups * n;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
         x += (size_t)gridDim.x * blockDim.x) {
        const int32_t g = (int32_t)(x / n), i = (int32_t)(x % n);
        const u32x4 u = philox((uint32_t)i, 0u, (uint32_t)t, (kTagInit << 24) | (uint32_t)(g + gbase), key0, key1);
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
    if (kind == 0) return H > kByteLaneMaxH ? sweep_wide_smem_bytes(n, cfg, false) : sweep_ising_smem_bytes(n, H, cfg);
    if (kind == 2) return sweep_softmax_smem_bytes(n, H, cfg);
    return sweep_potts_smem_bytes(n, H, cfg);
}

cudaError_t launch_sweep(int kind, int rule, int32_t n, const int32_t *rp, const uint32_t *adj,
                         int32_t H, const pamc_params &p, int32_t t, int32_t slot, SchedView sv,
                         const uint64_t *tab, const int8_t *src, const int32_t *parent,
                         const int8_t *ncm_buf, const int32_t *ncm_idx, int8_t *dst,
                         int64_t *E_dst, const DevCtl *ctl, SweepCfg cfg, int64_t Wsum,
                         cudaStream_t st, uint32_t *gsp, int32_t rbase, bool nib) {
    if (kind == 0 && nib)
        return launch_sweep_ising_nib(rule, n, H, p, t, slot, sv, tab, src, parent, ncm_buf, ncm_idx, dst, E_dst,
                                      ctl, cfg, st, rbase);
    if (kind == 0 && H > kByteLaneMaxH)
        return launch_sweep_ising_wide(rule, n, rp, adj, H, p, t, slot, sv, tab, src, parent, ncm_buf, ncm_idx,
                                       dst, E_dst, ctl, cfg, st, gsp, rbase);
    if (kind == 0)
        return launch_sweep_ising(rule, n, rp, adj, H, p, t, slot, sv, tab, src, parent, ncm_buf,
                                  ncm_idx, dst, E_dst, ctl, cfg, st, gsp, rbase);
    if (kind == 2)
        return launch_sweep_softmax(n, rp, adj, H, p, t, slot, sv, tab, src, parent, ncm_idx, dst, E_dst, ctl,
                                    cfg, Wsum, st, rbase);
    return launch_sweep_potts(n, rp, adj, H, p, t, slot, sv, tab, src, parent, dst, E_dst, ctl, cfg, Wsum, st,
                              rbase);
}

cudaError_t launch_init(int kind, int32_t K, int32_t n, const int32_t *rp, const uint32_t *adj, int32_t R,
                        uint64_t seed, int32_t t, int only_if_restart, const DevCtl *ctl,
                        int64_t Wsum, int8_t *spins, int64_t *E, cudaStream_t st, int32_t rbase) {
    const size_t total = (size_t)((R + 3) / 4) * n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_init_spins<<<grid, 256, 0, st>>>(kind, K, n, R, (uint32_t)seed, (uint32_t)(seed >> 32), t,
                                        only_if_restart, ctl, spins, rbase / 4);
    k_energy<<<R, 256, 0, st>>>(kind, n, rp, adj, R, only_if_restart, ctl, Wsum, t, spins, E);
    return cudaGetLastError();
}

cudaError_t launch_energy(int kind, int32_t n, const int32_t *rp, const uint32_t *adj, int32_t R,
                          const DevCtl *ctl, int64_t Wsum, const int8_t *spins, int64_t *E, cudaStream_t st) {
    k_energy<<<R, 256, 0, st>>>(kind, n, rp, adj, R, 0, ctl, Wsum, 0, spins, E);
    return cudaGetLastError();
}

cudaError_t launch_init_spins(int kind, int32_t K, int32_t n, int32_t R, uint64_t seed, int32_t t,
                              int only_if_restart, const DevCtl *ctl, int8_t *spins, cudaStream_t st,
                              int32_t rbase) {
    const size_t total = (size_t)((R + 3) / 4) * n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_init_spins<<<grid, 256, 0, st>>>(kind, K, n, R, (uint32_t)seed, (uint32_t)(seed >> 32), t,
                                        only_if_restart, ctl, spins, rbase / 4);
    return cudaGetLastError();
}

}  // namespace pamc
