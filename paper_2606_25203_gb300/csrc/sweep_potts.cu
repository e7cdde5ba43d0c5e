// sweep_potts.cu -- S sweeps of the three-state Potts population (Max-3-Cut)
// with the cascaded sampler of Suppl. S3 (Eq. 6-8): with
// syn_c(k) = sum_j J_kj [sigma_j = c], label 0 iff u0 < T1(syn1-syn0, syn2-syn0),
// else label 1 iff u1 < T2(syn2-syn1), else label 2.
//
// Layout.  Four replicas form a group.  For every vertex the group keeps two
// one-hot words in shared memory: byte q of w0 (w1) is 1 iff replica q has
// label 0 (1).  A neighbour adds J to the byte lanes of both accumulators with
// one 64-bit shared load and two multiply-adds, on a bias of 128 per byte
// (bytes never carry since sum_j |J_kj| <= 127); syn2 = sum_j J_kj - syn0 -
// syn1.  Replica r's draws are words 2(r mod 2), 2(r mod 2)+1 of
// Philox(k, sweep, t, FLIP<<24 | r/2): two calls per group.  Levels of the
// (t, sweep) schedule give the exact sequential order.  The couplings come
// from the position-indexed ELL of the schedule when it exists, else from CSR.
//
// Lane pairs (PAIR, ELL rows): two lanes share a position.  Lane s runs the
// Philox call of replicas 2s and 2s + 1 and sums the coupling slots of its
// parity; one shuffle adds the two partial byte-lane sums (one of them
// carries the bias) and one more ORs the two halves of the new label word.
// The draws and decisions are those of the one-lane body.
#include "pamc_device.cuh"
#include "pamc_internal.h"

namespace pamc {

namespace {

__device__ __forceinline__ void potts_barrier(int id, int nthreads, int groups) {
    if (groups == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
}

// one-hot words of four byte labels (0..2)
__device__ __forceinline__ uint2 onehot(uint32_t labels) {
    return make_uint2(__vcmpeq4(labels, 0u) & 0x01010101u, __vcmpeq4(labels, 0x01010101u) & 0x01010101u);
}

// The sweeps of one CTA's replica groups (groups bid*gpc .. bid*gpc+gpc-1 of
// the instance), shared by the single-instance and the batched kernels.
template <bool ELLP, bool PAIR>
__device__ __forceinline__ void
potts_body(int32_t n, int32_t n_pad, const int32_t *__restrict__ rp, const uint32_t *__restrict__ adj,
           int32_t H, int32_t R, int32_t S, uint32_t key0, uint32_t key1, int32_t t, int32_t slot,
           const int32_t *__restrict__ sorder, const int32_t *__restrict__ slvl,
           const int32_t *__restrict__ snlev, const uint32_t *__restrict__ sell,
           const int2 *__restrict__ spos, int32_t W, const uint64_t *__restrict__ tab,
           const int8_t *__restrict__ src, const int32_t *__restrict__ parent, int8_t *__restrict__ dst,
           int64_t *__restrict__ E_dst, const DevCtl *__restrict__ ctl, int64_t Wsum, int gpc, int tpg,
           int32_t bid, int32_t gbase) {
    extern __shared__ __align__(16) uint8_t smem[];
    if (ctl->done) return;
    const int32_t W1 = 4 * H + 1;
    const uint64_t *T1 = tab;                            // [(a + 2H) * W1 + (b + 2H)], read through L1
    uint64_t *T2s = reinterpret_cast<uint64_t *>(smem);  // [c + 2H]
    uint2 *oh_all = reinterpret_cast<uint2 *>(smem + (((size_t)W1 * 8 + 15) & ~(size_t)15));
    unsigned long long *red = reinterpret_cast<unsigned long long *>(oh_all + (size_t)gpc * n_pad);
    for (int i = threadIdx.x; i < W1; i += blockDim.x) T2s[i] = tab[(size_t)W1 * W1 + i];
    for (int i = threadIdx.x; i < gpc * 4; i += blockDim.x) red[i] = 0ull;

    const int gl = threadIdx.x / tpg, li = threadIdx.x % tpg;
    const int32_t g = bid * gpc + gl;
    const int32_t gk = g + gbase;   // the group's index in the whole population keys its draws
    const int32_t r0 = g * 4;
    const bool active = r0 < R;
    uint2 *oh = oh_all + (size_t)gl * n_pad;

    if (active) {
        // NCM is not defined for Potts: slot r reads its resampling parent
        const int8_t *rows[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) rows[q] = (r0 + q < R) ? src + (size_t)parent[r0 + q] * n : nullptr;
        for (int32_t k = li; k < n; k += tpg) {
            uint32_t lab = 0x03030303u;   // padding replicas: no label
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (rows[q] != nullptr) lab = (lab & ~(0xFFu << (8 * q))) | ((uint32_t)(uint8_t)rows[q][k] << (8 * q));
            oh[k] = onehot(lab);
        }
    }
    __syncthreads();

    if (active) {
        const size_t ell_stride = (size_t)(((n + 31) >> 5) << 5) * W;
        for (int32_t sw = 0; sw < S; ++sw) {
            const size_t sb = (size_t)slot * S + sw;
            const int32_t *ord = sorder + sb * (size_t)n;
            const int32_t *lp = slvl + sb * (size_t)(n + 1);
            const uint32_t *es = ELLP ? sell + sb * ell_stride : nullptr;
            const int2 *pos = ELLP ? spos + sb * (size_t)n : nullptr;
            const int32_t L = snlev[sb];
            for (int32_t lev = 0; lev < L; ++lev) {
                const int32_t beg = lp[lev], end = lp[lev + 1];
                if constexpr (PAIR && ELLP) {
                    // every lane of the group runs the same passes (the
                    // shuffles need whole warps); a pair past the level's end
                    // works on its last position and writes nothing
                    const int sl = li & 1;
                    const int32_t half = tpg >> 1;
                    for (int32_t b = beg; b < end; b += half) {
                        const int32_t iv = b + (li >> 1);
                        const bool valid = iv < end;
                        const int32_t i = valid ? iv : end - 1;
                        const int2 pr = pos[i];
                        const uint32_t *ep = es + (size_t)(i >> 5) * 32 * W + (i & 31);
                        uint32_t ev[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) ev[q] = 2 * q + sl < W ? ep[(2 * q + sl) * 32] : 0u;
                        const int32_t k = pr.x & 0xFFFFFF;
                        const int32_t deg = (int32_t)((uint32_t)pr.x >> 24);
                        const int32_t jsum = pr.y;
                        const u32x4 u = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t,
                                               (kTagFlip << 24) | (uint32_t)(2 * gk + sl), key0, key1);
                        uint32_t A0 = sl ? 0u : 0x80808080u, A1 = sl ? 0u : 0x80808080u;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const uint2 o = oh[ev[q] & 0xFFFFFFu];
                            const uint32_t J = (uint32_t)((int32_t)ev[q] >> 24);
                            A0 += o.x * J;
                            A1 += o.y * J;
                        }
                        for (int32_t b0 = 16; b0 < deg; b0 += 4) {   // W >= deg rounded up to 4
                            const uint32_t ew0 = ep[(b0 + sl) * 32], ew1 = ep[(b0 + 2 + sl) * 32];
                            const uint2 o0 = oh[ew0 & 0xFFFFFFu], o1 = oh[ew1 & 0xFFFFFFu];
                            const uint32_t J0 = (uint32_t)((int32_t)ew0 >> 24), J1 = (uint32_t)((int32_t)ew1 >> 24);
                            A0 += o0.x * J0 + o1.x * J1;
                            A1 += o0.y * J0 + o1.y * J1;
                        }
                        A0 += __shfl_xor_sync(0xffffffffu, A0, 1);
                        A1 += __shfl_xor_sync(0xffffffffu, A1, 1);
                        uint32_t lab = 0u;
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const int q = 2 * sl + j;
                            uint32_t c = 3u;   // padding replicas: no label
                            if (r0 + q < R) {
                                const int32_t s0 = (int32_t)((A0 >> (8 * q)) & 0xFFu) - 128;
                                const int32_t s1 = (int32_t)((A1 >> (8 * q)) & 0xFFu) - 128;
                                const int32_t s2 = jsum - s0 - s1;
                                const uint64_t t1 = __ldg(&T1[(size_t)(s1 - s0 + 2 * H) * W1 + (s2 - s0 + 2 * H)]);
                                const uint32_t w0 = j ? u.z : u.x, w1 = j ? u.w : u.y;
                                if ((uint64_t)w0 < t1) c = 0u;
                                else if ((uint64_t)w1 < T2s[s2 - s1 + 2 * H]) c = 1u;
                                else c = 2u;
                            }
                            lab |= c << (8 * q);
                        }
                        lab |= __shfl_xor_sync(0xffffffffu, lab, 1);
                        const uint2 nw = onehot(lab), old = oh[k];
                        if (valid && sl == 0 && (nw.x != old.x || nw.y != old.y)) oh[k] = nw;
                    }
                    potts_barrier(1 + gl, tpg, gpc);
                    continue;
                }
                for (int32_t i = beg + li; i < end; i += tpg) {
                    uint32_t A0 = 0x80808080u, A1 = 0x80808080u;
                    int32_t k, jsum;
                    u32x4 ua, ub;
                    if (ELLP) {
                        // the record, then up to sixteen coupling words in flight while
                        // the two Philox calls run (padding slots: coupling 0)
                        const int2 pr = pos[i];
                        const uint32_t *ep = es + (size_t)(i >> 5) * 32 * W + (i & 31);
                        uint32_t ev[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) ev[q] = q < W ? ep[q * 32] : 0u;
                        k = pr.x & 0xFFFFFF;
                        const int32_t deg = (int32_t)((uint32_t)pr.x >> 24);
                        jsum = pr.y;
                        ua = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t, (kTagFlip << 24) | (uint32_t)(2 * gk),
                                    key0, key1);
                        ub = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t, (kTagFlip << 24) | (uint32_t)(2 * gk + 1),
                                    key0, key1);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const uint2 o = oh[ev[q] & 0xFFFFFFu];
                            const uint32_t J = (uint32_t)((int32_t)ev[q] >> 24);
                            A0 += o.x * J;
                            A1 += o.y * J;
                        }
                        for (int32_t b0 = 16; b0 < deg; b0 += 4) {
                            uint32_t ew[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) ew[q] = ep[(b0 + q) * 32];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const uint2 o = oh[ew[q] & 0xFFFFFFu];
                                const uint32_t J = (uint32_t)((int32_t)ew[q] >> 24);
                                A0 += o.x * J;
                                A1 += o.y * J;
                            }
                        }
                    } else {
                        k = ord[i] & 0xFFFFFF;
                        jsum = 0;
                        for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
                            const uint32_t a = adj[e];
                            const int32_t J = (int32_t)a >> 24;
                            const uint2 o = oh[a & 0xFFFFFFu];
                            A0 += o.x * (uint32_t)J;
                            A1 += o.y * (uint32_t)J;
                            jsum += J;
                        }
                        ua = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t, (kTagFlip << 24) | (uint32_t)(2 * gk),
                                    key0, key1);
                        ub = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t, (kTagFlip << 24) | (uint32_t)(2 * gk + 1),
                                    key0, key1);
                    }
                    const uint32_t u0[4] = {ua.x, ua.z, ub.x, ub.z};
                    const uint32_t u1[4] = {ua.y, ua.w, ub.y, ub.w};
                    uint32_t lab = 0x03030303u;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (r0 + q >= R) break;
                        const int32_t s0 = (int32_t)((A0 >> (8 * q)) & 0xFFu) - 128;
                        const int32_t s1 = (int32_t)((A1 >> (8 * q)) & 0xFFu) - 128;
                        const int32_t s2 = jsum - s0 - s1;
                        const uint64_t t1 = __ldg(&T1[(size_t)(s1 - s0 + 2 * H) * W1 + (s2 - s0 + 2 * H)]);
                        uint32_t c;
                        if ((uint64_t)u0[q] < t1) c = 0;
                        else if ((uint64_t)u1[q] < T2s[s2 - s1 + 2 * H]) c = 1;
                        else c = 2;
                        lab = (lab & ~(0xFFu << (8 * q))) | (c << (8 * q));
                    }
                    const uint2 nw = onehot(lab), old = oh[k];
                    if (nw.x != old.x || nw.y != old.y) oh[k] = nw;
                }
                potts_barrier(1 + gl, tpg, gpc);
            }
        }

        // energy from the definition, E = -sum_k syn_{sigma_k}(k) - W, and the write-back
        long long acc[4] = {0, 0, 0, 0};
        for (int32_t k = li; k < n; k += tpg) {
            uint32_t A0 = 0x80808080u, A1 = 0x80808080u;
            int32_t jsum = 0;
            for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
                const uint32_t a = adj[e];
                const int32_t J = (int32_t)a >> 24;
                const uint2 o = oh[a & 0xFFFFFFu];
                A0 += o.x * (uint32_t)J;
                A1 += o.y * (uint32_t)J;
                jsum += J;
            }
            const uint2 ok = oh[k];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t s0 = (int32_t)((A0 >> (8 * q)) & 0xFFu) - 128;
                const int32_t s1 = (int32_t)((A1 >> (8 * q)) & 0xFFu) - 128;
                const bool l0 = (ok.x >> (8 * q)) & 1u, l1 = (ok.y >> (8 * q)) & 1u;
                const int32_t own = l0 ? s0 : (l1 ? s1 : jsum - s0 - s1);
                acc[q] += own;
                if (r0 + q < R) dst[(size_t)(r0 + q) * n + k] = (int8_t)(l0 ? 0 : (l1 ? 1 : 2));
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

template <bool ELLP, bool PAIR>
__global__ void __launch_bounds__(1024)
k_sweep_potts(int32_t n, int32_t n_pad, const int32_t *__restrict__ rp, const uint32_t *__restrict__ adj,
              int32_t H, int32_t R, int32_t S, uint32_t key0, uint32_t key1, int32_t t, int32_t slot,
              const int32_t *__restrict__ sorder, const int32_t *__restrict__ slvl,
              const int32_t *__restrict__ snlev, const uint32_t *__restrict__ sell,
              const int2 *__restrict__ spos, int32_t W, const uint64_t *__restrict__ tab,
              const int8_t *__restrict__ src, const int32_t *__restrict__ parent, int8_t *__restrict__ dst,
              int64_t *__restrict__ E_dst, const DevCtl *__restrict__ ctl, int64_t Wsum, int gpc, int tpg,
              int32_t gbase) {
    potts_body<ELLP, PAIR>(n, n_pad, rp, adj, H, R, S, key0, key1, t, slot, sorder, slvl, snlev, sell, spos, W,
                           tab, src, parent, dst, E_dst, ctl, Wsum, gpc, tpg, blockIdx.x, gbase);
}

// Many Max-3-Cut instances in one launch: CTA b works on instance items[b].x,
// its local block items[b].y; the member's step index comes from its device
// controller (ctl->t), which picks the double-buffered labels and energies
// and the schedule slot; steps at or past t_end do nothing.
template <bool ELLP>
__global__ void __launch_bounds__(1024)
k_sweep_potts_batched(const SweepDesc *__restrict__ descs, const int2 *__restrict__ items, int gpc, int tpg) {
    const int2 it = items[blockIdx.x];
    const SweepDesc &d = descs[it.x];
    const DevCtl *ctl = d.ctl;
    const int32_t t = ctl->t;
    if (t >= d.t_end) return;
    potts_body<ELLP, false>(d.n, d.n_pad, d.rp, d.adj, d.H, d.R, d.S, d.K.k0[0], d.K.k1[0], t, t % d.slots, d.sorder,
                     d.slvl, d.snlev, d.sell, d.spos, d.W, d.tab, d.sp[t & 1], d.parent, d.sp[(t + 1) & 1],
                     d.en[(t + 1) & 1], ctl, d.Wsum, gpc, tpg, it.y, d.gbase);
}

}  // namespace

size_t sweep_potts_smem_bytes(int32_t n, int32_t H, SweepCfg cfg) {
    const int32_t n_pad = (n + 3) & ~3;
    return (((size_t)(4 * H + 1) * 8 + 15) & ~(size_t)15) + (size_t)cfg.groups_per_cta * n_pad * 8 +
           (size_t)cfg.groups_per_cta * 4 * 8;
}

cudaError_t launch_sweep_potts(int32_t n, const int32_t *rp, const uint32_t *adj, int32_t H, const pamc_params &p,
                               int32_t t, int32_t slot, SchedView sv, const uint64_t *tab, const int8_t *src,
                               const int32_t *parent, int8_t *dst, int64_t *E_dst, const DevCtl *ctl,
                               SweepCfg cfg, int64_t Wsum, cudaStream_t st, int32_t rbase) {
    const int32_t groups = (p.R + 3) / 4;
    const int gpc = cfg.groups_per_cta, tpg = cfg.warps_per_group * 32;
    const size_t smem = sweep_potts_smem_bytes(n, H, cfg);
    const int grid = (groups + gpc - 1) / gpc;
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    const bool ell = sv.ell != nullptr;
    const bool pair = ell && cfg.lanes_per_vertex == 2;   // lane pairs: ELL rows only
    cudaError_t err;
#define PAMC_POTTS(EL, PA)                                                                                        \
    do {                                                                                                          \
        err = allow_dynamic_smem(k_sweep_potts<EL, PA>, smem);                                                    \
        if (err != cudaSuccess) return err;                                                                       \
        k_sweep_potts<EL, PA><<<grid, gpc * tpg, smem, st>>>(                                                     \
            n, (n + 3) & ~3, rp, adj, H, p.R, p.sweeps, k0, k1, t, slot, sv.order, sv.lvl_ptr, sv.nlev,           \
            EL ? sv.ell : nullptr, EL ? sv.pos : nullptr, EL ? sv.W : 0, tab, src, parent, dst, E_dst, ctl, Wsum, \
            gpc, tpg, rbase / 4);                                                                                 \
    } while (0)
    if (pair) PAMC_POTTS(true, true);
    else if (ell) PAMC_POTTS(true, false);
    else PAMC_POTTS(false, false);
#undef PAMC_POTTS
    return cudaGetLastError();
}

}  // namespace pamc

namespace pamc {

cudaError_t launch_sweep_potts_batched(bool ell, const SweepDesc *descs, const int2 *items, int32_t nitems,
                                       int32_t n_max, SweepCfg cfg, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const int gpc = cfg.groups_per_cta, tpg = cfg.warps_per_group * 32;
    const size_t smem = sweep_potts_smem_bytes(n_max, 127, cfg);
    cudaError_t err;
    if (ell) {
        err = allow_dynamic_smem(k_sweep_potts_batched<true>, smem);
        if (err != cudaSuccess) return err;
        k_sweep_potts_batched<true><<<nitems, gpc * tpg, smem, st>>>(descs, items, gpc, tpg);
    } else {
        err = allow_dynamic_smem(k_sweep_potts_batched<false>, smem);
        if (err != cudaSuccess) return err;
        k_sweep_potts_batched<false><<<nitems, gpc * tpg, smem, st>>>(descs, items, gpc, tpg);
    }
    return cudaGetLastError();
}

}  // namespace pamc
