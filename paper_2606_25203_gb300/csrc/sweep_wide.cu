// sweep_wide.cu -- S single-spin sweeps of an Ising population whose field
// range does not fit a byte lane (Eq. 3-4 for couplings with
// 127 < max_k sum_j |J_kj| <= 32767, |J| <= 127 each: weighted or hub-heavy
// graphs).
//
// Layout.  A replica group (the four replicas of one Philox4x32-10 call)
// keeps two 32-bit words per vertex: word x holds replicas 0 and 1 in its
// 16-bit lanes (bit 0 and bit 16), word y replicas 2 and 3.  A neighbour adds
// J to both lanes of each word with one multiply-add per word on a bias of
// 2^15 per lane; a lane never carries into its neighbour because
// sum_j |J_kj| <= 32767, so lane q holds 32768 + sum_j J_kj [s_j = +1] and
// h_q + H = 2 * lane_q + H - 65536 - sum_j J_kj indexes the threshold table
// (2H + 1 entries, read from device memory through the read-only cache).  The
// words sit in shared memory (8n bytes a group) or, for groups that do not
// fit, in a device buffer of the caller's.  Levels of the (t, sweep) schedule
// give the exact sequential order, as for the byte-lane sweep.
#include <cstring>

#include "pamc_device.cuh"
#include "pamc_internal.h"

namespace pamc {

namespace {

// Philox draws with the round keys precomputed (kernel parameter space).
struct KeysPreW {
    const PhiloxKeys &K;
    __device__ __forceinline__ u32x4 operator()(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) const {
        return philox_rk(c0, c1, c2, c3, K);
    }
};

__device__ __forceinline__ void wide_barrier(int id, int nthreads, int groups) {
    if (groups == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
}

// New spin bits (bit 0 / bit 16 of each word) from the lane accumulators.
template <int RULE>
__device__ __forceinline__ uint2 wide_decide(uint2 A, int32_t c0, const u32x4 &u, uint2 old,
                                             const uint64_t *__restrict__ tab, int32_t H) {
    const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
    uint32_t nb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t acc = q < 2 ? A.x : A.y, ow = q < 2 ? old.x : old.y;
        const int sh = 16 * (q & 1);
        const int32_t idx = 2 * (int32_t)((acc >> sh) & 0xFFFFu) + c0;   // h + H
        if (RULE == 0) {
            nb[q] = (uint64_t)uw[q] < __ldg(&tab[idx]) ? 1u : 0u;
        } else {
            const uint32_t s = (ow >> sh) & 1u;
            const int32_t ix = s ? idx : 2 * H - idx;                     // s*h + H
            nb[q] = ((uint64_t)uw[q] < __ldg(&tab[ix])) ? (s ^ 1u) : s;
        }
    }
    return make_uint2(nb[0] | (nb[1] << 16), nb[2] | (nb[3] << 16));
}

template <bool ELLP, int RULE, bool GSP>
__global__ void __launch_bounds__(1024) k_sweep_ising_wide(SweepDesc d, int gpc, int tpg) {
    extern __shared__ __align__(16) uint8_t smem[];
    const DevCtl *ctl = d.ctl;
    if (ctl->done) return;
    const int32_t n = d.n, n_pad = d.n_pad, H = d.H, R = d.R, S = d.S, W = d.W;
    uint2 *words_all = reinterpret_cast<uint2 *>(smem);
    unsigned long long *red = reinterpret_cast<unsigned long long *>(words_all + (GSP ? 0 : (size_t)gpc * n_pad));
    for (int i = threadIdx.x; i < gpc * 4; i += blockDim.x) red[i] = 0ull;

    const int gl = threadIdx.x / tpg, li = threadIdx.x % tpg;
    const int32_t g = blockIdx.x * gpc + gl;
    const int32_t r0 = g * 4;
    const bool active = r0 < R;
    // flips of replicas 0..3 counted at bits 0, 16, 1, 17 (below): those of
    // the replicas r0 + q < R
    const int32_t nlive = R - r0;
    const uint32_t live = nlive >= 4 ? 0x00030003u : nlive == 3 ? 0x00010003u : nlive == 2 ? 0x00010001u
                          : nlive == 1 ? 0x1u : 0u;
    uint2 *sp = GSP ? reinterpret_cast<uint2 *>(d.gsp) + (size_t)g * n_pad : words_all + (size_t)gl * n_pad;

    if (active) {
        // slot r reads the NCM output if the cluster move rewrote it, else its
        // resampling parent (the replica copy of the population step)
        const int8_t *rows[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int32_t r = r0 + q;
            if (r < R) {
                const int32_t m = d.ncm_idx[r];
                rows[q] = m >= 0 ? d.ncm_buf + (size_t)m * n : d.src + (size_t)d.parent[r] * n;
            } else {
                rows[q] = nullptr;
            }
        }
        for (int32_t k = li; k < n; k += tpg) {
            uint32_t b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = rows[q] != nullptr && rows[q][k] > 0 ? 1u : 0u;
            sp[k] = make_uint2(b[0] | (b[1] << 16), b[2] | (b[3] << 16));
        }
    }
    __syncthreads();

    if (active) {
        const size_t ell_stride = (size_t)(((n + 31) >> 5) << 5) * W;
        const uint32_t ctr3 = (kTagFlip << 24) | (uint32_t)(g + d.gbase);
        const KeysPreW draw{d.K};
        uint32_t nflip = 0;
        for (int32_t sw = 0; sw < S; ++sw) {
            const size_t sb = (size_t)d.slot * S + sw;
            const int32_t *ord = d.sorder + sb * (size_t)n;
            const int32_t *lp = d.slvl + sb * (size_t)(n + 1);
            const uint32_t *es = ELLP ? d.sell + sb * ell_stride : nullptr;
            const int2 *pos = ELLP ? d.spos + sb * (size_t)n : nullptr;
            const int32_t L = d.snlev[sb];
            for (int32_t lev = 0; lev < L; ++lev) {
                const int32_t beg = lp[lev], end = lp[lev + 1];
                for (int32_t i = beg + li; i < end; i += tpg) {
                    uint2 A = make_uint2(0x80008000u, 0x80008000u);
                    int32_t k, jsum;
                    if (ELLP) {
                        const int2 pr = pos[i];
                        k = pr.x & 0xFFFFFF;
                        const int32_t deg = (int32_t)((uint32_t)pr.x >> 24);
                        jsum = pr.y;
                        const uint32_t *ep = es + (size_t)(i >> 5) * 32 * W + (i & 31);
                        for (int32_t s = 0; s < deg; ++s) {
                            const uint32_t e = ep[(size_t)s * 32];
                            const uint2 w = sp[e & 0xFFFFFFu];
                            const uint32_t J = (uint32_t)((int32_t)e >> 24);
                            A.x += w.x * J;
                            A.y += w.y * J;
                        }
                    } else {
                        k = ord[i] & 0xFFFFFF;
                        jsum = 0;
                        for (int32_t e = d.rp[k]; e < d.rp[k + 1]; ++e) {
                            const uint32_t a = d.adj[e];
                            const int32_t J = (int32_t)a >> 24;
                            const uint2 w = sp[a & 0xFFFFFFu];
                            A.x += w.x * (uint32_t)J;
                            A.y += w.y * (uint32_t)J;
                            jsum += J;
                        }
                    }
                    const u32x4 u = draw((uint32_t)k, (uint32_t)sw, (uint32_t)d.t, ctr3);
                    const uint2 old = sp[k];
                    const uint2 nw = wide_decide<RULE>(A, H - 65536 - jsum, u, old, d.tab, H);
                    if (nw.x != old.x || nw.y != old.y) {
                        sp[k] = nw;
                        nflip += __popc(((nw.x ^ old.x) | ((nw.y ^ old.y) << 1)) & live);
                    }
                }
                wide_barrier(1 + gl, tpg, gpc);
            }
        }
        {   // the launch's flips into the controller's counter (every lane of the warp)
            unsigned long long v = nflip;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0 && v != 0ull)
                atomicAdd(reinterpret_cast<unsigned long long *>(&const_cast<DevCtl *>(ctl)->sweep_flips), v);
        }
        // energy from the definition, E = -1/2 sum_k s_k h_k, and the write-back
        long long acc[4] = {0, 0, 0, 0};
        for (int32_t k = li; k < n; k += tpg) {
            uint2 A = make_uint2(0x80008000u, 0x80008000u);
            int32_t jsum = 0;
            for (int32_t e = d.rp[k]; e < d.rp[k + 1]; ++e) {
                const uint32_t a = d.adj[e];
                const int32_t J = (int32_t)a >> 24;
                const uint2 w = sp[a & 0xFFFFFFu];
                A.x += w.x * (uint32_t)J;
                A.y += w.y * (uint32_t)J;
                jsum += J;
            }
            const uint2 wk = sp[k];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t av = q < 2 ? A.x : A.y, ow = q < 2 ? wk.x : wk.y;
                const int sh = 16 * (q & 1);
                const int32_t h = 2 * ((int32_t)((av >> sh) & 0xFFFFu) - 32768) - jsum;
                const int32_t sv = ((ow >> sh) & 1u) ? 1 : -1;
                acc[q] += (long long)sv * h;
                if (r0 + q < R) d.dst[(size_t)(r0 + q) * n + k] = (int8_t)sv;
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
    if (active && li < 4 && r0 + li < R) d.E_dst[r0 + li] = -((long long)red[gl * 4 + li] / 2);
}

}  // namespace

size_t sweep_wide_smem_bytes(int32_t n, SweepCfg cfg, bool global_spins) {
    const int32_t n_pad = (n + 3) & ~3;
    return (global_spins ? 0 : (size_t)cfg.groups_per_cta * n_pad * 8) + (size_t)cfg.groups_per_cta * 4 * 8;
}

cudaError_t launch_sweep_ising_wide(int rule, int32_t n, const int32_t *rp, const uint32_t *adj, int32_t H,
                                    const pamc_params &p, int32_t t, int32_t slot, SchedView sv,
                                    const uint64_t *tab, const int8_t *src, const int32_t *parent,
                                    const int8_t *ncm_buf, const int32_t *ncm_idx, int8_t *dst, int64_t *E_dst,
                                    const DevCtl *ctl, SweepCfg cfg, cudaStream_t st, uint32_t *gsp,
                                    int32_t rbase) {
    const int32_t groups = (p.R + 3) / 4;
    const int gpc = cfg.groups_per_cta, tpg = cfg.warps_per_group * 32;
    SweepDesc d;
    memset(&d, 0, sizeof(d));
    d.rp = rp; d.adj = adj; d.sorder = sv.order; d.slvl = sv.lvl_ptr; d.snlev = sv.nlev; d.sell = sv.ell;
    d.spos = sv.pos; d.tab = tab; d.src = src; d.parent = parent; d.ncm_buf = ncm_buf; d.ncm_idx = ncm_idx;
    d.dst = dst; d.E_dst = E_dst; d.ctl = ctl; d.n = n; d.n_pad = (n + 3) & ~3; d.H = H; d.R = p.R;
    d.S = p.sweeps; d.t = t; d.slot = slot; d.W = sv.W; d.K = make_philox_keys(p.seed); d.gsp = gsp;
    d.gbase = rbase / 4;
    const bool g = gsp != nullptr, ell = sv.ell != nullptr;
    const size_t smem = sweep_wide_smem_bytes(n, cfg, g);
    const int grid = (groups + gpc - 1) / gpc;
    cudaError_t err;
#define PAMC_WIDE(EL, RU, GS)                                                              \
    do {                                                                                   \
        err = allow_dynamic_smem(k_sweep_ising_wide<EL, RU, GS>, smem);                    \
        if (err != cudaSuccess) return err;                                                \
        k_sweep_ising_wide<EL, RU, GS><<<grid, gpc * tpg, smem, st>>>(d, gpc, tpg);        \
    } while (0)
    if (ell) {
        if (rule == 0) { if (g) PAMC_WIDE(true, 0, true); else PAMC_WIDE(true, 0, false); }
        else { if (g) PAMC_WIDE(true, 1, true); else PAMC_WIDE(true, 1, false); }
    } else {
        if (rule == 0) { if (g) PAMC_WIDE(false, 0, true); else PAMC_WIDE(false, 0, false); }
        else { if (g) PAMC_WIDE(false, 1, true); else PAMC_WIDE(false, 1, false); }
    }
#undef PAMC_WIDE
    return cudaGetLastError();
}

}  // namespace pamc
