// sweep_softmax.cu -- S sweeps of the K-state Potts population (Max-K-Cut)
// with the softmax noisy-argmax update of Sec. III.F (Eq. 8-9):
//   P_c = exp(beta syn_c) / sum_m exp(beta syn_m),  syn_c(k) = sum_j J_kj [sigma_j = c],
//   sigma_k <- argmax_c (P_c - gamma U_c),           U_c uniform on [0, 1).
// The choice is made in binary32 with round-to-nearest operations in a fixed
// order: d_c = max_m syn_m - syn_c, e_c = (float) exp(-beta d_c) from a table
// of det_exp values, S = e_0 + ... + e_{K-1}, P_c = e_c / S,
// U_c = (float) u_c * 2^-32, v_c = P_c - gamma U_c, the first maximal c wins.
//
// Layout.  Four replicas form a group; their labels sit in shared memory as
// one 32-bit word per vertex, one byte (0..K-1) per replica.  For label c the
// four replicas' syn_c are accumulated at once: a neighbour adds J to byte q
// of A_c when replica q's neighbour has label c (a byte-wise compare of the
// neighbour's word with c, times J), on a bias of 128 per byte; bytes never
// carry since sum_j |J_kj| <= 127.  The draws of replica r at vertex k are
// words c mod 4 of Philox(k, sweep, t, FLIP<<24 | (r * ceil(K/4) + c/4)).
// Levels of the (t, sweep) schedule give the exact sequential order, as for
// the Ising sweep.
//
// Quads (QUAD): four lanes share a position, lane q deciding replica q.  Each
// lane sums every fourth coupling of the row (one of them carries the bias);
// two shuffles per label add the partial byte-lane sums, two more OR the new
// label bytes.  The draws and decisions are those of the one-lane body.
#include "pamc_device.cuh"
#include "pamc_internal.h"

namespace pamc {

namespace {

constexpr int kMaxK = 8;

__device__ __forceinline__ void softmax_barrier(int id, int nthreads, int groups) {
    if (groups == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
}

template <bool QUAD>
__global__ void __launch_bounds__(1024)
k_sweep_softmax(int32_t n, int32_t n_pad, const int32_t *__restrict__ rp, const uint32_t *__restrict__ adj,
                int32_t H, int32_t K, float gamma, int32_t R, int32_t S, uint32_t key0, uint32_t key1,
                int32_t t, int32_t slot, const int32_t *__restrict__ sorder, const int32_t *__restrict__ slvl,
                const int32_t *__restrict__ snlev, const float *__restrict__ tab,
                const int8_t *__restrict__ src, const int32_t *__restrict__ parent,
                const int32_t *__restrict__ ncm_idx, int8_t *__restrict__ dst, int64_t *__restrict__ E_dst,
                const DevCtl *__restrict__ ctl, int64_t Wsum, int gpc, int tpg, int32_t rbase) {
    extern __shared__ __align__(16) uint8_t smem[];
    if (ctl->done) return;
    const int tabn = 2 * H + 1;
    float *tab_s = reinterpret_cast<float *>(smem);
    uint32_t *spins_all = reinterpret_cast<uint32_t *>(smem + (((size_t)tabn * 4 + 15) & ~(size_t)15));
    unsigned long long *red = reinterpret_cast<unsigned long long *>(spins_all + (size_t)gpc * n_pad);
    for (int i = threadIdx.x; i < tabn; i += blockDim.x) tab_s[i] = tab[i];
    for (int i = threadIdx.x; i < gpc * 4; i += blockDim.x) red[i] = 0ull;

    const int gl = threadIdx.x / tpg, li = threadIdx.x % tpg;
    const int32_t g = blockIdx.x * gpc + gl;
    const int32_t r0 = g * 4;
    const bool active = r0 < R;
    uint32_t *sp = spins_all + (size_t)gl * n_pad;
    const int32_t nb = (K + 3) / 4;
    (void)ncm_idx;

    if (active) {
        const int8_t *rows[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int32_t r = r0 + q;
            // NCM is not defined for Potts, so slot r always reads its parent
            rows[q] = (r < R) ? src + (size_t)parent[r] * n : nullptr;
        }
        for (int32_t k = li; k < n; k += tpg) {
            uint32_t w = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (rows[q] != nullptr) w |= (uint32_t)(uint8_t)rows[q][k] << (8 * q);
            sp[k] = w;
        }
    }
    __syncthreads();

    if (active) {
        for (int32_t sw = 0; sw < S; ++sw) {
            const size_t sb = (size_t)slot * S + sw;
            const int32_t *ord = sorder + sb * (size_t)n;
            const int32_t *lp = slvl + sb * (size_t)(n + 1);
            const int32_t L = snlev[sb];
            for (int32_t lev = 0; lev < L; ++lev) {
                const int32_t beg = lp[lev], end = lp[lev + 1];
                if constexpr (QUAD) {
                    // every lane of the group runs the same passes (the
                    // shuffles need whole warps); a quad past the level's end
                    // works on its last position and writes nothing
                    const int qq = li & 3;
                    const int32_t quarter = tpg >> 2;
                    for (int32_t b0 = beg; b0 < end; b0 += quarter) {
                        const int32_t iv = b0 + (li >> 2);
                        const bool valid = iv < end;
                        const int32_t k = ord[valid ? iv : end - 1] & 0xFFFFFF;
                        uint32_t A[kMaxK];
#pragma unroll
                        for (int c = 0; c < kMaxK; ++c) A[c] = qq == 0 ? 0x80808080u : 0u;
                        for (int32_t e = rp[k] + qq; e < rp[k + 1]; e += 4) {
                            const uint32_t a = adj[e];
                            const uint32_t J = (uint32_t)((int32_t)a >> 24);
                            const uint32_t w = sp[a & 0xFFFFFFu];
#pragma unroll
                            for (int c = 0; c < kMaxK; ++c)
                                if (c < K) A[c] += (__vcmpeq4(w, 0x01010101u * (uint32_t)c) & 0x01010101u) * J;
                        }
#pragma unroll
                        for (int c = 0; c < kMaxK; ++c)
                            if (c < K) {   // K is the same for every lane
                                A[c] += __shfl_xor_sync(0xffffffffu, A[c], 1);
                                A[c] += __shfl_xor_sync(0xffffffffu, A[c], 2);
                            }
                        uint32_t lab = 0u;
                        const int32_t r = r0 + qq;
                        if (r < R) {
                            int32_t syn[kMaxK];
                            int32_t smax = -1000;
#pragma unroll
                            for (int c = 0; c < kMaxK; ++c) {
                                syn[c] = (int32_t)((A[c] >> (8 * qq)) & 0xFFu) - 128;
                                if (c < K) smax = max(smax, syn[c]);
                            }
                            float ev[kMaxK];
                            float Ssum = 0.0f;
#pragma unroll
                            for (int c = 0; c < kMaxK; ++c) {
                                ev[c] = c < K ? tab_s[smax - syn[c]] : 0.0f;
                                if (c < K) Ssum = __fadd_rn(Ssum, ev[c]);
                            }
                            uint32_t u[kMaxK];
#pragma unroll
                            for (int b = 0; b < kMaxK / 4; ++b) {
                                if (b < nb) {
                                    const u32x4 x = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t,
                                                           (kTagFlip << 24) | (uint32_t)((r + rbase) * nb + b), key0,
                                                           key1);
                                    u[4 * b] = x.x; u[4 * b + 1] = x.y; u[4 * b + 2] = x.z; u[4 * b + 3] = x.w;
                                } else {
                                    u[4 * b] = u[4 * b + 1] = u[4 * b + 2] = u[4 * b + 3] = 0u;
                                }
                            }
                            int32_t best = 0;
                            float vbest = 0.0f;
#pragma unroll
                            for (int c = 0; c < kMaxK; ++c) {
                                if (c < K) {
                                    const float P = __fdiv_rn(ev[c], Ssum);
                                    const float U = __fmul_rn(__uint2float_rn(u[c]), 0x1p-32f);
                                    const float v = __fsub_rn(P, __fmul_rn(gamma, U));
                                    if (c == 0 || v > vbest) { vbest = v; best = c; }
                                }
                            }
                            lab = (uint32_t)best << (8 * qq);
                        }
                        lab |= __shfl_xor_sync(0xffffffffu, lab, 1);
                        lab |= __shfl_xor_sync(0xffffffffu, lab, 2);
                        if (valid && qq == 0 && lab != sp[k]) sp[k] = lab;
                    }
                    softmax_barrier(1 + gl, tpg, gpc);
                    continue;
                }
                for (int32_t i = beg + li; i < end; i += tpg) {
                    const int32_t k = ord[i] & 0xFFFFFF;
                    uint32_t A[kMaxK];
#pragma unroll
                    for (int c = 0; c < kMaxK; ++c) A[c] = 0x80808080u;
                    for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
                        const uint32_t a = adj[e];
                        const uint32_t J = (uint32_t)((int32_t)a >> 24);
                        const uint32_t w = sp[a & 0xFFFFFFu];
#pragma unroll
                        for (int c = 0; c < kMaxK; ++c)
                            if (c < K) A[c] += (__vcmpeq4(w, 0x01010101u * (uint32_t)c) & 0x01010101u) * J;
                    }
                    const uint32_t old = sp[k];
                    uint32_t nw = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int32_t r = r0 + q;
                        if (r >= R) break;
                        int32_t syn[kMaxK];
                        int32_t smax = -1000;
#pragma unroll
                        for (int c = 0; c < kMaxK; ++c) {
                            syn[c] = (int32_t)((A[c] >> (8 * q)) & 0xFFu) - 128;
                            if (c < K) smax = max(smax, syn[c]);
                        }
                        float ev[kMaxK];
                        float Ssum = 0.0f;
#pragma unroll
                        for (int c = 0; c < kMaxK; ++c) {
                            ev[c] = c < K ? tab_s[smax - syn[c]] : 0.0f;
                            if (c < K) Ssum = __fadd_rn(Ssum, ev[c]);
                        }
                        uint32_t u[kMaxK];
#pragma unroll
                        for (int b = 0; b < kMaxK / 4; ++b) {
                            if (b < nb) {
                                const u32x4 x = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t,
                                                       (kTagFlip << 24) | (uint32_t)((r + rbase) * nb + b), key0, key1);
                                u[4 * b] = x.x; u[4 * b + 1] = x.y; u[4 * b + 2] = x.z; u[4 * b + 3] = x.w;
                            } else {
                                u[4 * b] = u[4 * b + 1] = u[4 * b + 2] = u[4 * b + 3] = 0u;
                            }
                        }
                        int32_t best = 0;
                        float vbest = 0.0f;
#pragma unroll
                        for (int c = 0; c < kMaxK; ++c) {
                            if (c < K) {
                                const float P = __fdiv_rn(ev[c], Ssum);
                                const float U = __fmul_rn(__uint2float_rn(u[c]), 0x1p-32f);
                                const float v = __fsub_rn(P, __fmul_rn(gamma, U));
                                if (c == 0 || v > vbest) { vbest = v; best = c; }
                            }
                        }
                        nw |= (uint32_t)best << (8 * q);
                    }
                    if (nw != old) sp[k] = nw;
                }
                softmax_barrier(1 + gl, tpg, gpc);
            }
        }

        // energy from the definition, E = -sum_k syn_{sigma_k}(k) - W, and the write-back
        long long acc[4] = {0, 0, 0, 0};
        for (int32_t k = li; k < n; k += tpg) {
            const uint32_t wk = sp[k];
            uint32_t A = 0x80808080u;
            for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
                const uint32_t a = adj[e];
                const uint32_t J = (uint32_t)((int32_t)a >> 24);
                A += (__vcmpeq4(sp[a & 0xFFFFFFu], wk) & 0x01010101u) * J;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc[q] += (long long)((int32_t)((A >> (8 * q)) & 0xFFu) - 128);
                if (r0 + q < R) dst[(size_t)(r0 + q) * n + k] = (int8_t)((wk >> (8 * q)) & 0xFFu);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            long long v = acc[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&red[gl * 4 + q], (unsigned long long)v);
        }
    }
    __syncthreads();
    if (active && li < 4 && r0 + li < R) E_dst[r0 + li] = -(long long)red[gl * 4 + li] - Wsum;
}

}  // namespace

size_t sweep_softmax_smem_bytes(int32_t n, int32_t H, SweepCfg cfg) {
    const int32_t n_pad = (n + 3) & ~3;
    return (((size_t)(2 * H + 1) * 4 + 15) & ~(size_t)15) + (size_t)cfg.groups_per_cta * n_pad * 4 +
           (size_t)cfg.groups_per_cta * 4 * 8;
}

cudaError_t launch_sweep_softmax(int32_t n, const int32_t *rp, const uint32_t *adj, int32_t H,
                                 const pamc_params &p, int32_t t, int32_t slot, SchedView sv,
                                 const uint64_t *tab, const int8_t *src, const int32_t *parent,
                                 const int32_t *ncm_idx, int8_t *dst, int64_t *E_dst, const DevCtl *ctl,
                                 SweepCfg cfg, int64_t Wsum, cudaStream_t st, int32_t rbase) {
    const int32_t groups = (p.R + 3) / 4;
    const int gpc = cfg.groups_per_cta, tpg = cfg.warps_per_group * 32;
    const size_t smem = sweep_softmax_smem_bytes(n, H, cfg);
    const int grid = (groups + gpc - 1) / gpc;
    cudaError_t err;
#define PAMC_SOFTMAX(QU)                                                                                          \
    do {                                                                                                          \
        err = allow_dynamic_smem(k_sweep_softmax<QU>, smem);                                                      \
        if (err != cudaSuccess) return err;                                                                       \
        k_sweep_softmax<QU><<<grid, gpc * tpg, smem, st>>>(                                                       \
            n, (n + 3) & ~3, rp, adj, H, p.K, (float)p.gamma, p.R, p.sweeps, (uint32_t)p.seed,                    \
            (uint32_t)(p.seed >> 32), t, slot, sv.order, sv.lvl_ptr, sv.nlev, reinterpret_cast<const float *>(tab), \
            src, parent, ncm_idx, dst, E_dst, ctl, Wsum, gpc, tpg, rbase);                                        \
    } while (0)
    if (cfg.lanes_per_vertex == 4) PAMC_SOFTMAX(true);   // quads: four lanes a position
    else PAMC_SOFTMAX(false);
#undef PAMC_SOFTMAX
    return cudaGetLastError();
}

}  // namespace pamc
