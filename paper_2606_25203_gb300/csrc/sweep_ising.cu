// sweep_ising.cu -- S single-spin sweeps of the Ising population per
// temperature step (Eq. 3-4: heat-bath s_k = +1 iff u < T(h_k); Metropolis
// flip iff u < T_M(2 s_k h_k)), the hot loop of Algorithm 1.
//
// Layout.  A replica group (the 4 replicas that share one Philox4x32-10 call
// per vertex visit) keeps its spins in shared memory as one 32-bit word per
// vertex with one BYTE per replica (0 or 1).  A neighbour's contribution to
// the four fields is then a single word added to (or subtracted from) a
// biased accumulator A (one multiply-add: A += word_j * J_kj) whose byte q
// holds 128 + sum_j J_kj [s_j = +1], so that
//     h_q + H = 2 * byte_q(A) + c0,   c0 = H - 256 - sum_j J_kj
// indexes the threshold table directly.  Bytes never carry or borrow because
// sum_j |J_kj| <= 127.  A neighbour costs one global load (position-indexed
// ELL, batches of four in flight), one shared load and one multiply-add.
//
// Order.  Vertices of one level of the (t, sweep) schedule are pairwise
// uncoupled; levels run in order with a named barrier per replica group, which
// reproduces the sequential sweep exactly.
//
// Two ways of keeping the fields.  Pull (any H <= 127, any schedule, several
// lanes per vertex): a visit sums its neighbours' spin words as above.  Push
// (H <= 63, position-indexed ELL, one lane per vertex): byte q of a vertex's
// word holds replica q's spin in bit 7 and its biased field
// 64 + sum_j J_kj [s_j = +1] (in [1, 127]) in bits 0..6, computed once per
// launch from the CSR.  A visit reads its own word only; a flip adds
// (up - down) * J_jk to each neighbour's word -- the incrementally maintained
// fields of Eq. 3.  The record and first four couplings of the next position
// are loaded one iteration ahead as in the pull model, so a flip pushes
// without waiting.  Two vertices of a level may share
// a neighbour, so the updates are shared-memory atomics; 32-bit modular
// addition is exact because every byte of every intermediate word is the
// field byte of some configuration and stays in [1, 127].
#include <cstdlib>

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

// Spin flips of a launch (replicas whose spin changed at a visit), summed per
// warp into the controller's counter; every lane of the warp calls it.
// The spin bits (bit 8q of a word) of the replicas r0 + q < R: the lanes of
// a ragged last group that hold no replica are left out of the flip count.
__device__ __forceinline__ uint32_t live_byte_lanes(int32_t r0, int32_t R) {
    const int32_t v = R - r0;
    return v >= 4 ? 0x01010101u : v <= 0 ? 0u : 0x01010101u & ((1u << (8 * v)) - 1u);
}

__device__ __forceinline__ void count_flips(uint32_t nflip, const DevCtl *ctl) {
    unsigned long long v = nflip;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0ull)
        atomicAdd(reinterpret_cast<unsigned long long *>(&const_cast<DevCtl *>(ctl)->sweep_flips), v);
}

// Philox draws with the round keys precomputed (kernel parameter space) or
// advanced on the fly from the seed (batched launches, where the key differs
// per instance and would otherwise sit in local memory).
struct KeysPre {
    const PhiloxKeys &K;
    __device__ __forceinline__ u32x4 operator()(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) const {
        return philox_rk(c0, c1, c2, c3, K);
    }
};
struct KeysSeed {
    uint32_t k0, k1;
    __device__ __forceinline__ u32x4 operator()(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) const {
        return philox(c0, c1, c2, c3, k0, k1);
    }
};

// New four-replica spin word from the byte-lane field accumulator A (byte q =
// 128 + sum_j J_kj [s_j = +1]), c0 = H - 256 - sum_j J_kj, the draws u and the
// old word: heat-bath s = +1 iff u < T(h); Metropolis flip iff u < T_M(2 s h).
template <int RULE>
__device__ __forceinline__ uint32_t ising_decide(uint32_t A, int32_t c0, const u32x4 &u, uint32_t old,
                                                 const uint64_t *tab_s, int32_t H) {
    const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
    uint32_t nw = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // byte q of A, zero-extended (one byte permute)
        const int32_t idx = 2 * (int32_t)__byte_perm(A, 0u, 0x4440u + q) + c0;   // h + H
        if (RULE == 0) {
            nw |= ((uint64_t)uw[q] < tab_s[idx] ? 1u : 0u) << (8 * q);
        } else {
            const uint32_t s = (old >> (8 * q)) & 1u;
            const int32_t ix = s ? idx : 2 * H - idx;              // s*h + H
            nw |= (((uint64_t)uw[q] < tab_s[ix]) ? (s ^ 1u) : s) << (8 * q);
        }
    }
    return nw;
}

// The push model's decision: byte q of the vertex word F holds the spin of
// replica q in bit 7 and the biased field 64 + sum_j J_kj [s_j = +1] in bits
// 0..6; c0 = H - 128 - sum_j J_kj, so that 2 * field byte + c0 = h + H.
template <int RULE>
__device__ __forceinline__ uint32_t ising_decide_push(uint32_t F, int32_t c0, const u32x4 &u,
                                                      const uint64_t *tab_s, int32_t H) {
    const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
    uint32_t nw = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int32_t idx = 2 * (int32_t)((F >> (8 * q)) & 0x7Fu) + c0;   // h + H
        if (RULE == 0) {
            nw |= ((uint64_t)uw[q] < tab_s[idx] ? 1u : 0u) << (8 * q);
        } else {
            const uint32_t sq = (F >> (8 * q + 7)) & 1u;
            const int32_t ix = sq ? idx : 2 * H - idx;             // s*h + H
            nw |= (((uint64_t)uw[q] < tab_s[ix]) ? (sq ^ 1u) : sq) << (8 * q);
        }
    }
    return nw;
}

// Push-model sweeps of one CTA's replica groups (H <= 63, position-indexed
// ELL, one lane per vertex, S >= 1); same inputs, outputs and shared-memory
// layout as the pull body below, and bit-identical results.
template <int RULE, class KeyT>
__device__ __forceinline__ void
sweep_ising_push_body(int32_t n, int32_t n_pad, const int32_t *__restrict__ rp,
                      const uint32_t *__restrict__ adj, int32_t H, int32_t R, int32_t S, const KeyT &draw,
                      int32_t t, int32_t slot, const int32_t *__restrict__ slvl,
                      const int32_t *__restrict__ snlev, const uint32_t *__restrict__ sell,
                      const int2 *__restrict__ spos, int32_t W, const uint64_t *__restrict__ tab,
                      const int8_t *__restrict__ src, const int32_t *__restrict__ parent,
                      const int8_t *__restrict__ ncm_buf, const int32_t *__restrict__ ncm_idx,
                      int8_t *__restrict__ dst, int64_t *__restrict__ E_dst, const DevCtl *__restrict__ ctl,
                      int gpc, int tpg, int32_t bid, int32_t gbase = 0) {
    extern __shared__ __align__(16) uint8_t smem[];
    if (ctl->done) return;
    const int tabn = 2 * H + 1;
    uint64_t *tab_s = reinterpret_cast<uint64_t *>(smem);
    uint32_t *spins_all = reinterpret_cast<uint32_t *>(smem + (((size_t)tabn * 8 + 15) & ~(size_t)15));
    unsigned long long *red = reinterpret_cast<unsigned long long *>(spins_all + (size_t)gpc * n_pad);
    for (int i = threadIdx.x; i < tabn; i += blockDim.x) tab_s[i] = tab[i];
    for (int i = threadIdx.x; i < gpc * 4; i += blockDim.x) red[i] = 0ull;

    const int gl = threadIdx.x / tpg, li = threadIdx.x % tpg;
    const int32_t g = bid * gpc + gl;
    const int32_t r0 = g * 4;
    const bool active = r0 < R;
    const uint32_t live = live_byte_lanes(r0, R);
    uint32_t *sp = spins_all + (size_t)gl * n_pad;

    if (active) {
        // the replica copy of the population step (see the pull body): spin
        // bits and fields of each vertex straight from the source rows in
        // global memory, so that no thread reads a word another one writes
        const int8_t *rows[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int32_t r = r0 + q;
            if (r < R) {
                const int32_t m = ncm_idx[r];
                rows[q] = m >= 0 ? ncm_buf + (size_t)m * n : src + (size_t)parent[r] * n;
            } else {
                rows[q] = nullptr;
            }
        }
        auto bits = [&](int32_t j) {
            uint32_t w = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (rows[q] != nullptr) w |= (uint32_t)(rows[q][j] > 0) << (8 * q);
            return w;
        };
        for (int32_t k = li; k < n; k += tpg) {
            uint32_t A = 0x40404040u;
            for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
                const uint32_t a = adj[e];
                A += bits((int32_t)(a & 0xFFFFFFu)) * (uint32_t)((int32_t)a >> 24);
            }
            sp[k] = (bits(k) << 7) | A;
        }
    }
    __syncthreads();

    if (active) {
        const size_t ell_stride = (size_t)(((n + 31) >> 5) << 5) * W;
        const uint32_t ctr3 = (kTagFlip << 24) | (uint32_t)(g + gbase);
        uint32_t nflip = 0;
        for (int32_t sw = 0; sw < S; ++sw) {
            const size_t sb = (size_t)slot * S + sw;
            const int32_t *lp = slvl + sb * (size_t)(n + 1);
            const uint32_t *es = sell + sb * ell_stride;
            const int2 *pos = spos + sb * (size_t)n;
            const int32_t L = snlev[sb];
            // the record and the first four couplings of a position are loaded
            // one iteration ahead -- for a level's first position before the
            // previous level's barrier, from a clamped position (they do not
            // depend on spins); a flip pushes along them
            int2 pr = make_int2(0, 0);
            uint32_t e4[4] = {0u, 0u, 0u, 0u};
            auto fetch = [&](int32_t i, int2 &r, uint32_t (&e)[4]) {
                r = pos[i];
                const uint32_t *ep = es + (size_t)(i >> 5) * 32 * W + (i & 31);
#pragma unroll
                for (int q = 0; q < 4; ++q) e[q] = ep[q * 32];
            };
            if (L > 0) fetch(min(li, n - 1), pr, e4);
            for (int32_t lev = 0; lev < L; ++lev) {
                const int32_t beg = lp[lev], end = lp[lev + 1];
                int32_t i = beg + li;
                while (i < end) {
                    const int32_t inext = i + tpg;
                    int2 prn = make_int2(0, 0);
                    uint32_t e4n[4] = {0u, 0u, 0u, 0u};
                    if (inext < end) fetch(inext, prn, e4n);
                    const int32_t k = pr.x & 0xFFFFFF;
                    const uint32_t F = sp[k];
                    const u32x4 u = draw((uint32_t)k, (uint32_t)sw, (uint32_t)t, ctr3);
                    const uint32_t old = (F >> 7) & 0x01010101u;
                    const uint32_t nw = ising_decide_push<RULE>(F, H - 128 - pr.y, u, tab_s, H);
                    const uint32_t fl = nw ^ old;
                    if (fl != 0u) {
                        sp[k] = F ^ (fl << 7);
                        nflip += __popc(fl & live);
                        // per byte +1 (up) or -1 (down), mod 2^32, times J_jk
                        const uint32_t delta = (nw & fl) - (old & fl);
                        const int32_t deg = (int32_t)((uint32_t)pr.x >> 24);
#pragma unroll
                        for (int q = 0; q < 4; ++q)   // padding slots: vertex 0, coupling 0
                            if (q < deg) atomicAdd(&sp[e4[q] & 0xFFFFFFu], delta * (uint32_t)((int32_t)e4[q] >> 24));
                        if (deg > 4) {
                            const uint32_t *ep = es + (size_t)(i >> 5) * 32 * W + (i & 31);
                            for (int32_t sl = 4; sl < deg; ++sl) {
                                const uint32_t e = ep[(size_t)sl * 32];
                                atomicAdd(&sp[e & 0xFFFFFFu], delta * (uint32_t)((int32_t)e >> 24));
                            }
                        }
                    }
                    i = inext;
                    pr = prn;
#pragma unroll
                    for (int q = 0; q < 4; ++q) e4[q] = e4n[q];
                }
                if (lev + 1 < L) fetch(min(end + li, n - 1), pr, e4);
                group_barrier(1 + gl, tpg, gpc);
            }
        }

        count_flips(nflip, ctl);
        // energy E = -1/2 sum_k s_k h_k from the fields (by position over the
        // last sweep's records, which carry sum_j J_kj), and the write-back
        int32_t acc[4] = {0, 0, 0, 0};
        const int2 *pos = spos + ((size_t)slot * S + (S - 1)) * (size_t)n;
        for (int32_t i = li; i < n; i += tpg) {
            const int2 p0 = pos[i];
            const uint32_t F = sp[p0.x & 0xFFFFFF];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t h = 2 * ((int32_t)((F >> (8 * q)) & 0x7Fu) - 64) - p0.y;
                acc[q] += ((F >> (8 * q + 7)) & 1u) ? h : -h;
            }
        }
        for (int32_t k = li; k < n; k += tpg) {
            const uint32_t w = sp[k];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (r0 + q < R) dst[(size_t)(r0 + q) * n + k] = ((w >> (8 * q + 7)) & 1u) ? 1 : -1;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            long long v = acc[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&red[gl * 4 + q], (unsigned long long)v);
        }
    }
    __syncthreads();
    if (active && li < 4 && r0 + li < R) E_dst[r0 + li] = -((long long)red[gl * 4 + li] / 2);
}

// Row i of a position-indexed ELL block of width W: lanes of a warp read
// consecutive words (slot s of position i at (i & ~31) * W + 32 s + (i & 31)),
// with 32-bit offset arithmetic (n W < 2^32: n < 2^24, W < 256).
__device__ __forceinline__ const uint32_t *ell_row(const uint32_t *es, int32_t i, int32_t W) {
    return es + ((uint32_t)(i & ~31) * (uint32_t)W + (uint32_t)(i & 31));
}

// The sweep of one CTA's replica groups (groups bid*gpc .. bid*gpc+gpc-1 of
// the instance), shared by the single-instance and the batched kernels.  With
// LPV > 1 (position-indexed ELL only; LPV a power of two up to 32) LPV lanes share a vertex: lane sub takes
// the coupling slots sub, sub + LPV, ...; the byte-lane partial sums add up
// exactly under XOR shuffles (plain 32-bit addition), and every lane of the
// group runs the same iterations so that the shuffles always converge.
template <bool ELLP, int RULE, int LPV, class KeyT, bool GSP = false, int WC = 0>
__device__ __forceinline__ void
sweep_ising_body(int32_t n, int32_t n_pad, const int32_t *__restrict__ rp,
                 const uint32_t *__restrict__ adj, int32_t H, int32_t R, int32_t S, const KeyT &draw,
                 int32_t t, int32_t slot, const int32_t *__restrict__ sorder,
                 const int32_t *__restrict__ slvl, const int32_t *__restrict__ snlev,
                 const uint32_t *__restrict__ sell, const int2 *__restrict__ spos, int32_t W,
                 const uint64_t *__restrict__ tab, const int8_t *__restrict__ src,
                 const int32_t *__restrict__ parent, const int8_t *__restrict__ ncm_buf,
                 const int32_t *__restrict__ ncm_idx, int8_t *__restrict__ dst,
                 int64_t *__restrict__ E_dst, const DevCtl *__restrict__ ctl, int gpc, int tpg,
                 int32_t bid, uint32_t *__restrict__ gspins = nullptr, int32_t gbase = 0) {
    // WC > 0: the ELL width, known at compile time (4: every row in the first
    // four slots, the torus; 8, 12, 16: sparse graphs of low degree)
    if constexpr (WC > 0) W = WC;
    extern __shared__ __align__(16) uint8_t smem[];
    if (ctl->done) return;
    const int tabn = 2 * H + 1;
    uint64_t *tab_s = reinterpret_cast<uint64_t *>(smem);
    // the groups' spin words: shared memory, or (GSP) the caller's device
    // buffer of n_pad words per group, for groups that do not fit on chip or
    // where more groups per SM pay; the level barriers order both alike
    uint32_t *spins_all = reinterpret_cast<uint32_t *>(smem + (((size_t)tabn * 8 + 15) & ~(size_t)15));
    unsigned long long *red = reinterpret_cast<unsigned long long *>(spins_all + (GSP ? 0 : (size_t)gpc * n_pad));
    for (int i = threadIdx.x; i < tabn; i += blockDim.x) tab_s[i] = tab[i];
    for (int i = threadIdx.x; i < gpc * 4; i += blockDim.x) red[i] = 0ull;

    const int gl = threadIdx.x / tpg, li = threadIdx.x % tpg;
    const int32_t g = bid * gpc + gl;
    const int32_t r0 = g * 4;
    const bool active = r0 < R;
    const uint32_t live = live_byte_lanes(r0, R);
    uint32_t *sp = GSP ? gspins + (size_t)g * n_pad : spins_all + (size_t)gl * n_pad;

    if (active) {
        // slot r reads the NCM output if the cluster move rewrote it, else
        // its resampling parent (the replica copy of the population step)
        const int8_t *rows[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int32_t r = r0 + q;
            if (r < R) {
                const int32_t m = ncm_idx[r];
                rows[q] = m >= 0 ? ncm_buf + (size_t)m * n : src + (size_t)parent[r] * n;
            } else {
                rows[q] = nullptr;
            }
        }
        for (int32_t k = li; k < n; k += tpg) {
            uint32_t w = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (rows[q] != nullptr) w |= (uint32_t)(rows[q][k] > 0) << (8 * q);
            sp[k] = w;
        }
    }
    __syncthreads();

    if (active) {
        const size_t ell_stride = (size_t)(((n + 31) >> 5) << 5) * W;
        const uint32_t ctr3 = (kTagFlip << 24) | (uint32_t)(g + gbase);
        uint32_t nflip = 0;
        for (int32_t sw = 0; sw < S; ++sw) {
            const size_t sb = (size_t)slot * S + sw;
            const int32_t *ord = sorder + sb * (size_t)n;
            const int32_t *lp = slvl + sb * (size_t)(n + 1);
            const uint32_t *es = ELLP ? sell + sb * ell_stride : nullptr;
            const int2 *pos = ELLP ? spos + sb * (size_t)n : nullptr;
            const int32_t L = snlev[sb];
            if constexpr (ELLP && LPV > 1) {
                // lane sub of a vertex takes the slots sub + LPV q; the record
                // and the first eight slots of a pass are loaded ahead, for a
                // level's first pass before the previous level's barrier
                // (from a clamped position: they do not depend on spins)
                const int32_t vl = li / LPV, sub = li % LPV, vpi = tpg / LPV;
                int2 pr;
                uint32_t e8[8];
                auto fetch = [&](int32_t i) {
                    pr = pos[i];
                    const uint32_t *ep = ell_row(es, i, W);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int32_t sl = sub + q * LPV;   // slots >= deg hold coupling 0
                        e8[q] = sl < W ? ep[(size_t)sl * 32] : 0u;
                    }
                };
                if (L > 0) fetch(min(vl, n - 1));
                for (int32_t lev = 0; lev < L; ++lev) {
                    const int32_t beg = lp[lev], end = lp[lev + 1];
                    for (int32_t base = beg; base < end; base += vpi) {   // uniform over the group
                        // idle lanes take a clamped position too: a whole row of
                        // one vertex, so that its sum indexes the table in range
                        const bool act = base + vl < end;
                        const int32_t ic = min(base + vl, n - 1);
                        if (base != beg) fetch(ic);
                        const int32_t k = pr.x & 0xFFFFFF;
                        const int32_t deg = (int32_t)((uint32_t)pr.x >> 24);
                        const u32x4 u = draw((uint32_t)k, (uint32_t)sw, (uint32_t)t, ctr3);
                        uint32_t Ap = 0u;
#pragma unroll
                        for (int q = 0; q < 8; ++q) Ap += sp[e8[q] & 0xFFFFFFu] * (uint32_t)((int32_t)e8[q] >> 24);
                        if (8 * LPV < deg) {
                            const uint32_t *ep = ell_row(es, ic, W);
                            for (int32_t s0 = sub + 8 * LPV; s0 < deg; s0 += 8 * LPV) {
                                uint32_t ev[8];
#pragma unroll
                                for (int q = 0; q < 8; ++q) {
                                    const int32_t sl = s0 + q * LPV;
                                    ev[q] = sl < W ? ep[(size_t)sl * 32] : 0u;
                                }
#pragma unroll
                                for (int q = 0; q < 8; ++q)
                                    Ap += sp[ev[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ev[q] >> 24);
                            }
                        }
#pragma unroll
                        for (int o = 1; o < LPV; o <<= 1) Ap += __shfl_xor_sync(0xffffffffu, Ap, o);
                        const uint32_t old = sp[k];
                        const uint32_t nw = ising_decide<RULE>(0x80808080u + Ap, H - 256 - pr.y, u, old, tab_s, H);
                        // every lane has read sp[k] before any lane of the group writes it
                        __syncwarp();
                        if (act && sub == 0 && nw != old) {
                            sp[k] = nw;
                            nflip += __popc((nw ^ old) & live);
                        }
                    }
                    if (lev + 1 < L) fetch(min(end + vl, n - 1));
                    group_barrier(1 + gl, tpg, gpc);
                }
                continue;
            }
            // ELL path: the record and the first four neighbour words of a
            // position are loaded one iteration ahead -- for a level's first
            // position before the previous level's barrier (they do not
            // depend on spins), so the wait overlaps the barrier
            int2 pr = make_int2(0, 0);
            uint32_t e4[4] = {0u, 0u, 0u, 0u};
            int32_t end = 0;
            if (ELLP && L > 0) {
                // unconditional, from a clamped position: whether it is used is
                // decided once the level's bounds are known
                const int32_t i0 = min(li, n - 1);
                pr = pos[i0];
                const uint32_t *ep = ell_row(es, i0, W);
#pragma unroll
                for (int q = 0; q < 4; ++q) e4[q] = ep[q * 32];
            }
            for (int32_t lev = 0; lev < L; ++lev) {
                const int32_t beg = lp[lev];
                end = lp[lev + 1];
                int32_t i = beg + li;
                while (i < end) {
                    const int32_t inext = i + tpg;
                    int2 prn = make_int2(0, 0);
                    uint32_t e4n[4] = {0u, 0u, 0u, 0u};
                    if (ELLP && inext < end) {
                        prn = pos[inext];
                        const uint32_t *epn = ell_row(es, inext, W);
#pragma unroll
                        for (int q = 0; q < 4; ++q) e4n[q] = epn[q * 32];
                    }
                    // A: byte q = 128 + sum_j J_kj [s_j = +1] of replica q
                    uint32_t A = 0x80808080u;
                    int32_t k, jsum;
                    u32x4 u;
                    if (ELLP) {
                        const uint32_t a0 = (uint32_t)pr.x;
                        k = (int32_t)(a0 & 0xFFFFFFu);
                        const int32_t deg = (int32_t)(a0 >> 24);
                        jsum = pr.y;
                        // the next neighbour words are requested before the draw is
                        // computed, so that the Philox rounds overlap their latency
                        if (W <= 4) {   // every neighbour word is already in registers
#pragma unroll
                            for (int q = 0; q < 4; ++q)   // padding slots: coupling 0
                                A += sp[e4[q] & 0xFFFFFFu] * (uint32_t)((int32_t)e4[q] >> 24);
                            u = draw((uint32_t)k, (uint32_t)sw, (uint32_t)t, ctr3);
                        } else if constexpr (WC > 0 && WC <= 16) {
                        const uint32_t *ep = ell_row(es, i, W) + 4 * 32;
                        // rows of at most sixteen slots (compile-time width):
                        // the words beyond the first four in blocks of four,
                        // all in flight before the draw (a level's positions
                        // are grouped by degree, so a warp's lanes mostly
                        // agree on how many blocks they need)
                        uint32_t ev[4], ew[4], ex[4];
                        if (deg > 4) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) ev[q] = (4 + q < W) ? ep[q * 32] : 0u;
                        }
                        if (deg > 8) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) ew[q] = (8 + q < W) ? ep[(4 + q) * 32] : 0u;
                        }
                        if (deg > 12) {
#pragma unroll
                            for (int q = 0; q < 4; ++q) ex[q] = (12 + q < W) ? ep[(8 + q) * 32] : 0u;
                        }
                        u = draw((uint32_t)k, (uint32_t)sw, (uint32_t)t, ctr3);
#pragma unroll
                        for (int q = 0; q < 4; ++q)   // padding slots: coupling 0
                            A += sp[e4[q] & 0xFFFFFFu] * (uint32_t)((int32_t)e4[q] >> 24);
                        if (deg > 4) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                A += sp[ev[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ev[q] >> 24);
                        }
                        if (deg > 8) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                A += sp[ew[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ew[q] >> 24);
                        }
                        if (deg > 12) {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                A += sp[ex[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ex[q] >> 24);
                        }
                        } else {
                        const uint32_t *ep = ell_row(es, i, W) + 4 * 32;
                        // up to sixteen more neighbour words in flight before the draw
                        uint32_t ev[8], ew[8];
                        if (deg > 4) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) ev[q] = (4 + q < W) ? ep[q * 32] : 0u;
                        }
                        if (deg > 12) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) ew[q] = (12 + q < W) ? ep[(8 + q) * 32] : 0u;
                        }
                        u = draw((uint32_t)k, (uint32_t)sw, (uint32_t)t, ctr3);
#pragma unroll
                        for (int q = 0; q < 4; ++q)   // padding slots: coupling 0
                            A += sp[e4[q] & 0xFFFFFFu] * (uint32_t)((int32_t)e4[q] >> 24);
                        if (deg > 4) {
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                A += sp[ev[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ev[q] >> 24);
                        }
                        if (deg > 12) {
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                A += sp[ew[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ew[q] >> 24);
                        }
                        for (int32_t b0 = 20; b0 < deg; b0 += 8) {
                            ep += (b0 == 20 ? 16 : 8) * 32;
#pragma unroll
                            for (int q = 0; q < 8; ++q) ev[q] = (b0 + q < W) ? ep[q * 32] : 0u;
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                A += sp[ev[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ev[q] >> 24);
                        }
                        }
                    } else {
                        k = ord[i] & 0xFFFFFF;
                        jsum = 0;
                        for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
                            const uint32_t a = adj[e];
                            const int32_t J = (int32_t)a >> 24;
                            A += sp[a & 0xFFFFFFu] * (uint32_t)J;
                            jsum += J;
                        }
                    }
                    if (!ELLP) u = draw((uint32_t)k, (uint32_t)sw, (uint32_t)t, ctr3);
                    const uint32_t old = sp[k];
                    const uint32_t nw = ising_decide<RULE>(A, H - 256 - jsum, u, old, tab_s, H);
                    if (nw != old) {
                        sp[k] = nw;
                        nflip += __popc((nw ^ old) & live);
                    }
                    i = inext;
                    pr = prn;
#pragma unroll
                    for (int q = 0; q < 4; ++q) e4[q] = e4n[q];
                }
                if (ELLP && lev + 1 < L) {   // the next level's first position (clamped, see above)
                    const int32_t i2 = min(end + li, n - 1);
                    pr = pos[i2];
                    const uint32_t *ep = ell_row(es, i2, W);
#pragma unroll
                    for (int q = 0; q < 4; ++q) e4[q] = ep[q * 32];
                }
                group_barrier(1 + gl, tpg, gpc);
            }
        }

        count_flips(nflip, ctl);
        // energy from the definition E = -1/2 sum_k s_k h_k (per thread at most
        // n / 32 vertices of |s h| <= 127 each: int32), and the write-back
        int32_t acc[4] = {0, 0, 0, 0};
        if (ELLP && S > 0) {
            // by position over the last sweep's ELL rows: coalesced loads that do
            // not depend on spins, the next position's issued one ahead
            const size_t sb = (size_t)slot * S + (S - 1);
            const uint32_t *es = sell + sb * ell_stride;
            const int2 *pos = spos + sb * (size_t)n;
            int2 pr = make_int2(0, 0);
            uint32_t e4[4] = {0u, 0u, 0u, 0u};
            auto fetch = [&](int32_t i) {
                pr = pos[i];
                const uint32_t *ep = ell_row(es, i, W);
#pragma unroll
                for (int q = 0; q < 4; ++q) e4[q] = q < W ? ep[q * 32] : 0u;
            };
            if (li < n) fetch(li);
            for (int32_t i = li; i < n; i += tpg) {
                const int2 p0 = pr;
                uint32_t A = 0x80808080u;
#pragma unroll
                for (int q = 0; q < 4; ++q) A += sp[e4[q] & 0xFFFFFFu] * (uint32_t)((int32_t)e4[q] >> 24);
                if (i + tpg < n) fetch(i + tpg);
                const int32_t deg = (int32_t)((uint32_t)p0.x >> 24);
                if (deg > 4) {
                    const uint32_t *ep = ell_row(es, i, W);
                    for (int32_t sl = 4; sl < deg; ++sl) {
                        const uint32_t e = ep[(size_t)sl * 32];
                        A += sp[e & 0xFFFFFFu] * (uint32_t)((int32_t)e >> 24);
                    }
                }
                const uint32_t w = sp[p0.x & 0xFFFFFF];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int32_t h = 2 * ((int32_t)((A >> (8 * q)) & 0xFFu) - 128) - p0.y;   // p0.y = sum_j J_kj
                    acc[q] += ((w >> (8 * q)) & 1u) ? h : -h;
                }
            }
            for (int32_t k = li; k < n; k += tpg) {
                const uint32_t w = sp[k];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (r0 + q < R) dst[(size_t)(r0 + q) * n + k] = ((w >> (8 * q)) & 1u) ? 1 : -1;
            }
        } else {
            for (int32_t k = li; k < n; k += tpg) {
                const uint32_t w = sp[k];
                uint32_t A = 0x80808080u;
                int32_t jsum = 0;
                for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
                    const uint32_t a = adj[e];
                    const int32_t J = (int32_t)a >> 24;
                    A += sp[a & 0xFFFFFFu] * (uint32_t)J;
                    jsum += J;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int32_t h = 2 * ((int32_t)((A >> (8 * q)) & 0xFFu) - 128) - jsum;
                    const int32_t sv = ((w >> (8 * q)) & 1u) ? 1 : -1;
                    acc[q] += sv * h;
                    if (r0 + q < R) dst[(size_t)(r0 + q) * n + k] = (int8_t)sv;
                }
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
    if (active && li < 4 && r0 + li < R) E_dst[r0 + li] = -((long long)red[gl * 4 + li] / 2);
}

template <bool ELLP, int RULE, int LPV, bool GSP = false, int WC = 0>
__global__ void __launch_bounds__(1024) k_sweep_ising(SweepDesc d, int gpc, int tpg) {
    sweep_ising_body<ELLP, RULE, LPV, KeysPre, GSP, WC>(d.n, d.n_pad, d.rp, d.adj, d.H, d.R, d.S, KeysPre{d.K}, d.t,
                                                    d.slot, d.sorder, d.slvl, d.snlev, d.sell, d.spos, d.W, d.tab,
                                                    d.src, d.parent, d.ncm_buf, d.ncm_idx, d.dst, d.E_dst, d.ctl, gpc,
                                                    tpg, blockIdx.x, d.gsp, d.gbase);
}

template <int RULE>
__global__ void __launch_bounds__(1024) k_sweep_ising_push(SweepDesc d, int gpc, int tpg) {
    sweep_ising_push_body<RULE>(d.n, d.n_pad, d.rp, d.adj, d.H, d.R, d.S, KeysPre{d.K}, d.t, d.slot, d.slvl,
                                d.snlev, d.sell, d.spos, d.W, d.tab, d.src, d.parent, d.ncm_buf, d.ncm_idx,
                                d.dst, d.E_dst, d.ctl, gpc, tpg, blockIdx.x, d.gbase);
}

// Many instances in one launch: CTA b works on instance items[b].x, its
// local block items[b].y.  Descriptors live in device memory and are read
// field by field (no local copy of the descriptor).  LPV > 1: lanes per
// vertex, as for one instance (ELL schedules only).
template <bool ELLP, int RULE, int LPV, bool GSP = false>
__global__ void __launch_bounds__(1024)
k_sweep_ising_batched(const SweepDesc *__restrict__ descs, const int2 *__restrict__ items, int gpc, int tpg) {
    const int2 it = items[blockIdx.x];
    const SweepDesc &d = descs[it.x];
    const DevCtl *ctl = d.ctl;
    const int32_t t = ctl->t;
    if (t >= d.t_end) return;
    const KeysSeed draw{d.K.k0[0], d.K.k1[0]};
    if constexpr (ELLP && LPV == 1 && !GSP) {
        if (d.push) {   // uniform over the CTA: one member per CTA
            sweep_ising_push_body<RULE>(d.n, d.n_pad, d.rp, d.adj, d.H, d.R, d.S, draw, t, t % d.slots, d.slvl,
                                        d.snlev, d.sell, d.spos, d.W, d.tab, d.sp[t & 1], d.parent, d.ncm_buf,
                                        d.ncm_idx, d.sp[(t + 1) & 1], d.en[(t + 1) & 1], ctl, gpc, tpg, it.y, d.gbase);
            return;
        }
    }
    sweep_ising_body<ELLP, RULE, LPV, KeysSeed, GSP>(d.n, d.n_pad, d.rp, d.adj, d.H, d.R, d.S, draw, t, t % d.slots,
                                                     d.sorder, d.slvl, d.snlev, d.sell, d.spos, d.W, d.tab,
                                                     d.sp[t & 1], d.parent, d.ncm_buf, d.ncm_idx, d.sp[(t + 1) & 1],
                                                     d.en[(t + 1) & 1], ctl, gpc, tpg, it.y, d.gsp, d.gbase);
}

}  // namespace

// Opt-in (PAMC_SWEEP_PUSH=1): on the low-degree instances measured (torus,
// average degree 5.7) the push sweep ran slower than the pull sweep, since a
// flip's updates are paid by every lane of its warp.
bool sweep_push_enabled() {
    const char *env = getenv("PAMC_SWEEP_PUSH");
    return env && env[0] == '1';
}

bool sweep_push_ok(int32_t H, int32_t S, bool ell, int lanes_per_vertex) {
    return ell && lanes_per_vertex == 1 && H <= 63 && S > 0 && sweep_push_enabled();
}

size_t sweep_ising_smem_bytes(int32_t n, int32_t H, SweepCfg cfg, bool global_spins) {
    const int32_t n_pad = (n + 3) & ~3;
    return (((size_t)(2 * H + 1) * 8 + 15) & ~(size_t)15) +
           (global_spins ? 0 : (size_t)cfg.groups_per_cta * n_pad * 4) + (size_t)cfg.groups_per_cta * 4 * 8;
}

cudaError_t launch_sweep_ising(int rule, int32_t n, const int32_t *rp, const uint32_t *adj,
                               int32_t H, const pamc_params &p, int32_t t, int32_t slot,
                               SchedView sv, const uint64_t *tab, const int8_t *src,
                               const int32_t *parent, const int8_t *ncm_buf,
                               const int32_t *ncm_idx, int8_t *dst, int64_t *E_dst,
                               const DevCtl *ctl, SweepCfg cfg, cudaStream_t st, uint32_t *gsp,
                               int32_t rbase) {
    const int32_t groups = (p.R + 3) / 4;
    const int gpc = cfg.groups_per_cta, tpg = cfg.warps_per_group * 32;
    SweepDesc d;
    d.rp = rp; d.adj = adj; d.sorder = sv.order; d.slvl = sv.lvl_ptr; d.snlev = sv.nlev; d.sell = sv.ell;
    d.spos = sv.pos; d.tab = tab; d.src = src; d.parent = parent; d.ncm_buf = ncm_buf; d.ncm_idx = ncm_idx;
    d.dst = dst; d.E_dst = E_dst; d.ctl = ctl; d.n = n; d.n_pad = (n + 3) & ~3; d.H = H; d.R = p.R;
    d.S = p.sweeps; d.t = t; d.slot = slot; d.W = sv.W; d.K = make_philox_keys(p.seed);
    d.gsp = gsp;
    d.gbase = rbase / 4;
    const size_t smem = sweep_ising_smem_bytes(n, H, cfg, gsp != nullptr);
    const int grid = (groups + gpc - 1) / gpc;
    const bool ell = sv.ell != nullptr;
    cudaError_t err = cudaSuccess;
#define PAMC_LAUNCH(EL, RU, LV)                                                                   \
    do {                                                                                          \
        err = allow_dynamic_smem(k_sweep_ising<EL, RU, LV>, smem);                                \
        if (err != cudaSuccess) return err;                                                       \
        k_sweep_ising<EL, RU, LV><<<grid, gpc * tpg, smem, st>>>(d, gpc, tpg);                    \
    } while (0)
#define PAMC_LAUNCH_WC(RU, WV)                                                                    \
    do {                                                                                          \
        err = allow_dynamic_smem(k_sweep_ising<true, RU, 1, false, WV>, smem);                    \
        if (err != cudaSuccess) return err;                                                       \
        k_sweep_ising<true, RU, 1, false, WV><<<grid, gpc * tpg, smem, st>>>(d, gpc, tpg);        \
    } while (0)
#define PAMC_LAUNCH_G(EL, RU)                                                                     \
    do {                                                                                          \
        err = allow_dynamic_smem(k_sweep_ising<EL, RU, 1, true>, smem);                           \
        if (err != cudaSuccess) return err;                                                       \
        k_sweep_ising<EL, RU, 1, true><<<grid, gpc * tpg, smem, st>>>(d, gpc, tpg);               \
    } while (0)
#define PAMC_LAUNCH_LPV(RU)                                                                       \
    do {                                                                                          \
        switch (lpv) {                                                                            \
        case 32: PAMC_LAUNCH(true, RU, 32); break;                                                \
        case 16: PAMC_LAUNCH(true, RU, 16); break;                                                \
        case 8: PAMC_LAUNCH(true, RU, 8); break;                                                  \
        case 4: PAMC_LAUNCH(true, RU, 4); break;                                                  \
        case 2: PAMC_LAUNCH(true, RU, 2); break;                                                  \
        default:                                                                                  \
            switch (sv.W) {                                                                       \
            case 4: PAMC_LAUNCH_WC(RU, 4); break;                                                 \
            case 8: PAMC_LAUNCH_WC(RU, 8); break;                                                 \
            case 12: PAMC_LAUNCH_WC(RU, 12); break;                                               \
            case 16: PAMC_LAUNCH_WC(RU, 16); break;                                               \
            default: PAMC_LAUNCH(true, RU, 1); break;                                             \
            }                                                                                     \
            break;                                                                                \
        }                                                                                         \
    } while (0)
    const int lpv = ell ? cfg.lanes_per_vertex : 1;
    if (gsp) {   // spin words in device memory: one lane per vertex
        if (ell) {
            if (rule == 0) PAMC_LAUNCH_G(true, 0); else PAMC_LAUNCH_G(true, 1);
        } else {
            if (rule == 0) PAMC_LAUNCH_G(false, 0); else PAMC_LAUNCH_G(false, 1);
        }
        return cudaGetLastError();
    }
    d.push = sweep_push_ok(H, p.sweeps, ell, lpv) ? 1 : 0;
    if (d.push) {
        if (rule == 0) {
            err = allow_dynamic_smem(k_sweep_ising_push<0>, smem);
            if (err != cudaSuccess) return err;
            k_sweep_ising_push<0><<<grid, gpc * tpg, smem, st>>>(d, gpc, tpg);
        } else {
            err = allow_dynamic_smem(k_sweep_ising_push<1>, smem);
            if (err != cudaSuccess) return err;
            k_sweep_ising_push<1><<<grid, gpc * tpg, smem, st>>>(d, gpc, tpg);
        }
        return cudaGetLastError();
    }
    if (ell) {
        if (rule == 0) PAMC_LAUNCH_LPV(0); else PAMC_LAUNCH_LPV(1);
    } else {
        if (rule == 0) PAMC_LAUNCH(false, 0, 1); else PAMC_LAUNCH(false, 1, 1);
    }
#undef PAMC_LAUNCH_LPV
#undef PAMC_LAUNCH_G
#undef PAMC_LAUNCH_WC
#undef PAMC_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_sweep_ising_batched(int rule, bool ell, const SweepDesc *descs, const int2 *items,
                                       int32_t nitems, int32_t n_max, SweepCfg cfg, cudaStream_t st,
                                       bool global_spins) {
    if (nitems <= 0) return cudaSuccess;
    const int gpc = cfg.groups_per_cta, tpg = cfg.warps_per_group * 32;
    const size_t smem = sweep_ising_smem_bytes(n_max, 127, cfg, global_spins);
    cudaError_t err = cudaSuccess;
    if (global_spins) {   // one lane per vertex
#define PAMC_LAUNCH_BG(EL, RU)                                                                        \
    do {                                                                                              \
        err = allow_dynamic_smem(k_sweep_ising_batched<EL, RU, 1, true>, smem);                       \
        if (err != cudaSuccess) return err;                                                           \
        k_sweep_ising_batched<EL, RU, 1, true><<<nitems, gpc * tpg, smem, st>>>(descs, items, gpc, tpg); \
    } while (0)
        if (ell) {
            if (rule == 0) PAMC_LAUNCH_BG(true, 0); else PAMC_LAUNCH_BG(true, 1);
        } else {
            if (rule == 0) PAMC_LAUNCH_BG(false, 0); else PAMC_LAUNCH_BG(false, 1);
        }
#undef PAMC_LAUNCH_BG
        return cudaGetLastError();
    }
#define PAMC_LAUNCH(EL, RU, LV)                                                                   \
    do {                                                                                          \
        err = allow_dynamic_smem(k_sweep_ising_batched<EL, RU, LV>, smem);                        \
        if (err != cudaSuccess) return err;                                                       \
        k_sweep_ising_batched<EL, RU, LV><<<nitems, gpc * tpg, smem, st>>>(descs, items, gpc, tpg); \
    } while (0)
#define PAMC_LAUNCH_LPV(RU)                                                                       \
    do {                                                                                          \
        switch (cfg.lanes_per_vertex) {                                                           \
        case 4: PAMC_LAUNCH(true, RU, 4); break;                                                  \
        case 2: PAMC_LAUNCH(true, RU, 2); break;                                                  \
        default: PAMC_LAUNCH(true, RU, 1); break;                                                 \
        }                                                                                         \
    } while (0)
    if (ell) {
        if (rule == 0) PAMC_LAUNCH_LPV(0); else PAMC_LAUNCH_LPV(1);
    } else {
        if (rule == 0) PAMC_LAUNCH(false, 0, 1); else PAMC_LAUNCH(false, 1, 1);
    }
#undef PAMC_LAUNCH_LPV
#undef PAMC_LAUNCH
    return cudaGetLastError();
}

}  // namespace pamc
