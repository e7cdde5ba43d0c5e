// sweep_nibble.cu -- the Ising sweep (Eq. 3-4) with EIGHT replicas per
// 32-bit word, for instances whose field range fits 4-bit lanes.
//
// Layout.  Nibble q of a vertex's word holds the spin of replica 8g + q of
// replica group g (1 = +1).  A neighbour costs one ELL word, one shared load
// and one multiply-add for eight replicas (twice the byte lanes' four), and a
// group's words take the same 4n bytes of shared memory for twice the
// replicas.
//
// Fixed bias (sum_j |J_kj| <= 7 for every vertex: the +-1 torus, graphs of
// degree <= 7; ELL width 4 or 8).  A = 0x88888888 + sum_j J_kj word_j has
// nibble q = 8 + sum_j J_kj [s_j = +1] in [1, 15]: no nibble carries or
// borrows, so h_q + H = 2 nibble_q(A) + c0, c0 = H - 16 - sum_j J_kj, indexes
// the threshold table as in the byte-lane kernel.
//
// Biased lanes (ELL width up to 16; sum |J| <= 15 over the slots 0..7 and
// over the slots 8..15 of every vertex: +-1 graphs of degree <= 16, such as
// sparse random graphs of mean degree 6).  With M the weight of the negative
// couplings of a half, A_half = M 0x11111111 + sum_{j in half} J_kj word_j
// has nibble q = N_q = sum_{J > 0} J [s_j = +1] + sum_{J < 0} |J| [s_j = -1]
// in [0, 15] (the satisfied weight of the half; every partial sum stays in
// range, so the word sums exactly), and h_q = 2 (N1_q + N2_q) - sum_j |J_kj|.
// The two halves are added in byte lanes (even and odd nibbles apart, sums
// <= 30), and h_q + H = 2 (N1_q + N2_q) + c0 with c0 = H - sum_j |J_kj|.  The
// per-vertex constants (M1 0x11111111, M2 0x11111111, c0) are computed once
// per instance.
//
// Draws.  Replica r uses word r mod 4 of Philox(k, sweep, t, FLIP<<24 | r/4)
// as everywhere else: the eight replicas of a word take two calls, of the
// four-replica groups 2g and 2g + 1 (offset by the population's group base),
// so the results are those of the byte-lane kernel bit for bit.
//
// Order: the (t, sweep) schedule's dependency levels with position-indexed
// ELL rows, one barrier per level, as in sweep_ising.cu.
#include <cstdlib>
#include <cstring>

#include "pamc_device.cuh"
#include "pamc_internal.h"

namespace pamc {

namespace {

// Philox draws with the round keys of the seed in kernel parameter space, or
// advanced from the seed (batched launches: the key differs per member).
struct NibKeys {
    const PhiloxKeys &K;
    __device__ __forceinline__ u32x4 operator()(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) const {
        return philox_rk(c0, c1, c2, c3, K);
    }
};
struct NibKeysSeed {
    uint32_t k0, k1;
    __device__ __forceinline__ u32x4 operator()(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) const {
        return philox(c0, c1, c2, c3, k0, k1);
    }
};

__device__ __forceinline__ void nib_barrier(int id, int nthreads, int groups) {
    if (groups == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
}

__device__ __forceinline__ const uint32_t *nib_ell_row(const uint32_t *es, int32_t i, int32_t W) {
    return es + ((uint32_t)(i & ~31) * (uint32_t)W + (uint32_t)(i & 31));
}

// New eight-replica word from the nibble accumulator A, c0 = H - 16 -
// sum_j J_kj, the draws of the two four-replica groups and the old word.
template <int RULE>
__device__ __forceinline__ uint32_t ising_decide8(uint32_t A, int32_t c0, const u32x4 &ua, const u32x4 &ub,
                                                  uint32_t old, const uint64_t *tab_s, int32_t H) {
    const uint32_t uw[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
    uint32_t nw = 0;
    // heat-bath: entry h + H = 2 nibble + c0 sits 16 * nibble bytes past
    // tab_s + c0, and 16 * nibble is nibble q of A moved to bits 4..7
    const char *tp = reinterpret_cast<const char *>(tab_s + c0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int32_t idx = 2 * (int32_t)((A >> (4 * q)) & 0xFu) + c0;   // h + H
        if (RULE == 0) {
            const uint32_t off = q == 0 ? (A << 4) & 0xF0u : (A >> (4 * q - 4)) & 0xF0u;
            const uint64_t T = *reinterpret_cast<const uint64_t *>(tp + off);
            nw |= ((uint64_t)uw[q] < T ? 1u : 0u) << (4 * q);
        } else {
            const uint32_t s = (old >> (4 * q)) & 1u;
            const int32_t ix = s ? idx : 2 * H - idx;              // s*h + H
            nw |= (((uint64_t)uw[q] < tab_s[ix]) ? (s ^ 1u) : s) << (4 * q);
        }
    }
    return nw;
}

// Biased lanes: the same from the byte-lane sums E (even nibbles: replica
// 2b in byte b) and O (odd nibbles: replica 2b + 1), each N1_q + N2_q in
// [0, 30], and c0 = H - sum_j |J_kj|.
template <int RULE>
__device__ __forceinline__ uint32_t ising_decide8b(uint32_t E, uint32_t O, int32_t c0, const u32x4 &ua,
                                                   const u32x4 &ub, uint32_t old, const uint64_t *tab_s,
                                                   int32_t H) {
    const uint32_t uw[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
    uint32_t nw = 0;
    // heat-bath: entry h + H = 2 N + c0 sits 16 N bytes past tab_s + c0
    const char *tp = reinterpret_cast<const char *>(tab_s + c0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t src = (q & 1) ? O : E;
        const int b = q >> 1;
        if (RULE == 0) {
            const uint32_t off = b == 0 ? (src << 4) & 0x1F0u : (src >> (8 * b - 4)) & 0x1F0u;
            const uint64_t T = *reinterpret_cast<const uint64_t *>(tp + off);
            nw |= ((uint64_t)uw[q] < T ? 1u : 0u) << (4 * q);
        } else {
            const int32_t idx = 2 * (int32_t)((src >> (8 * b)) & 0xFFu) + c0;   // h + H
            const uint32_t s = (old >> (4 * q)) & 1u;
            const int32_t ix = s ? idx : 2 * H - idx;                         // s*h + H
            nw |= (((uint64_t)uw[q] < tab_s[ix]) ? (s ^ 1u) : s) << (4 * q);
        }
    }
    return nw;
}

__device__ __forceinline__ void nib_halves(uint32_t A1, uint32_t A2, uint32_t &E, uint32_t &O) {
    E = (A1 & 0x0F0F0F0Fu) + (A2 & 0x0F0F0F0Fu);
    O = ((A1 >> 4) & 0x0F0F0F0Fu) + ((A2 >> 4) & 0x0F0F0F0Fu);
}

// The sweeps of one CTA's groups of eight (groups bid*gpc .. bid*gpc+gpc-1
// of the instance), shared by the single-instance and the batched kernels;
// WC = 0: the ELL width read at run time; BIASED: the biased lanes (width 4
// to 16, per-vertex constants d.nibc), else the fixed bias (width 4 or 8).
template <int RULE, int WC, bool BIASED, class KeyT>
__device__ __forceinline__ void
nib_body(const SweepDesc &d, const KeyT &draw, int32_t t, int32_t slot, const int8_t *__restrict__ src,
         int8_t *__restrict__ dst, int64_t *__restrict__ E_dst, int gpc, int tpg, int32_t bid) {
    extern __shared__ __align__(16) uint8_t smem[];
    const DevCtl *ctl = d.ctl;
    if (ctl->done) return;
    const int32_t n = d.n, n_pad = d.n_pad, H = d.H, R = d.R, S = d.S;
    const int32_t W = WC > 0 ? WC : d.W;
    const int tabn = 2 * H + 1;
    uint64_t *tab_s = reinterpret_cast<uint64_t *>(smem);
    uint32_t *spins_all = reinterpret_cast<uint32_t *>(smem + (((size_t)tabn * 8 + 15) & ~(size_t)15));
    unsigned long long *red = reinterpret_cast<unsigned long long *>(spins_all + (size_t)gpc * n_pad);
    for (int i = threadIdx.x; i < tabn; i += blockDim.x) tab_s[i] = d.tab[i];
    for (int i = threadIdx.x; i < gpc * 8; i += blockDim.x) red[i] = 0ull;

    const int gl = threadIdx.x / tpg, li = threadIdx.x % tpg;
    const int32_t g = bid * gpc + gl;   // group of eight replicas
    const int32_t r0 = g * 8;
    const bool active = r0 < R;
    // the spin bits (bit 4q) of the replicas r0 + q < R, for the flip count
    const uint32_t live = R - r0 >= 8 ? 0x11111111u : R - r0 <= 0 ? 0u : 0x11111111u & ((1u << (4 * (R - r0))) - 1u);
    uint32_t *sp = spins_all + (size_t)gl * n_pad;

    if (active) {
        // slot r reads the NCM output if the cluster move rewrote it, else its
        // resampling parent (the replica copy of the population step)
        const int8_t *rows[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int32_t r = r0 + q;
            if (r < R) {
                const int32_t m = d.ncm_idx[r];
                rows[q] = m >= 0 ? d.ncm_buf + (size_t)m * n : src + (size_t)d.parent[r] * n;
            } else {
                rows[q] = nullptr;
            }
        }
        for (int32_t k = li; k < n; k += tpg) {
            uint32_t w = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (rows[q] != nullptr) w |= (uint32_t)(rows[q][k] > 0) << (4 * q);
            sp[k] = w;
        }
    }
    __syncthreads();

    if (active) {
        const size_t ell_stride = (size_t)(((n + 31) >> 5) << 5) * W;
        const uint32_t ctrA = (kTagFlip << 24) | (uint32_t)(2 * g + d.gbase);
        const uint32_t ctrB = ctrA + 1u;
        uint32_t nflip = 0;
        for (int32_t sw = 0; sw < S; ++sw) {
            const size_t sb = (size_t)slot * S + sw;
            const int32_t *lp = d.slvl + sb * (size_t)(n + 1);
            const uint32_t *es = d.sell + sb * ell_stride;
            const int2 *pos = d.spos + sb * (size_t)n;
            const int32_t L = d.snlev[sb];
            // the record and the first four neighbour words of a position are
            // loaded one iteration ahead -- for a level's first position before
            // the previous level's barrier (they do not depend on spins)
            // (biased lanes: and the vertex's constants)
            int2 pr = make_int2(0, 0);
            uint32_t e4[4] = {0u, 0u, 0u, 0u};
            int4 nc = make_int4(0, 0, 0, 0);
            int32_t end = 0;
            if (L > 0) {
                const int32_t i0 = min(li, n - 1);
                pr = pos[i0];
                const uint32_t *ep = nib_ell_row(es, i0, W);
#pragma unroll
                for (int q = 0; q < 4; ++q) e4[q] = ep[q * 32];
                if constexpr (BIASED) nc = d.nibc[pr.x & 0xFFFFFF];
            }
            for (int32_t lev = 0; lev < L; ++lev) {
                const int32_t beg = lp[lev];
                end = lp[lev + 1];
                int32_t i = beg + li;
                while (i < end) {
                    const int32_t inext = i + tpg;
                    int2 prn = make_int2(0, 0);
                    uint32_t e4n[4] = {0u, 0u, 0u, 0u};
                    int4 ncn = make_int4(0, 0, 0, 0);
                    if (inext < end) {
                        prn = pos[inext];
                        const uint32_t *epn = nib_ell_row(es, inext, W);
#pragma unroll
                        for (int q = 0; q < 4; ++q) e4n[q] = epn[q * 32];
                        if constexpr (BIASED) ncn = d.nibc[prn.x & 0xFFFFFF];
                    }
                    const uint32_t a0 = (uint32_t)pr.x;
                    const int32_t k = (int32_t)(a0 & 0xFFFFFFu);
                    uint32_t A = BIASED ? (uint32_t)nc.x : 0x88888888u;
                    if (W > 4) {   // slots 4..7 (padding slots hold coupling 0)
                        const uint32_t *ep = nib_ell_row(es, i, W) + 4 * 32;
                        uint32_t ev[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) ev[q] = ep[q * 32];
#pragma unroll
                        for (int q = 0; q < 4; ++q) A += sp[ev[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ev[q] >> 24);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) A += sp[e4[q] & 0xFFFFFFu] * (uint32_t)((int32_t)e4[q] >> 24);
                    uint32_t A2 = 0u;
                    if constexpr (BIASED) {
                        // slots 8..15 into the second half, in blocks of four
                        // while the degree asks for them (levels are grouped
                        // by degree, so a warp's lanes mostly agree)
                        A2 = (uint32_t)nc.y;
                        const int32_t deg = (int32_t)(a0 >> 24);
                        if (W > 8 && deg > 8) {
                            const uint32_t *ep = nib_ell_row(es, i, W) + 8 * 32;
                            uint32_t ev[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) ev[q] = ep[q * 32];
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                A2 += sp[ev[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ev[q] >> 24);
                            if (W > 12 && deg > 12) {
#pragma unroll
                                for (int q = 0; q < 4; ++q) ev[q] = ep[(4 + q) * 32];
#pragma unroll
                                for (int q = 0; q < 4; ++q)
                                    A2 += sp[ev[q] & 0xFFFFFFu] * (uint32_t)((int32_t)ev[q] >> 24);
                            }
                        }
                    }
                    const u32x4 ua = draw((uint32_t)k, (uint32_t)sw, (uint32_t)t, ctrA);
                    const u32x4 ub = draw((uint32_t)k, (uint32_t)sw, (uint32_t)t, ctrB);
                    const uint32_t old = sp[k];
                    uint32_t nw;
                    if constexpr (BIASED) {
                        uint32_t E, O;
                        nib_halves(A, A2, E, O);
                        nw = ising_decide8b<RULE>(E, O, nc.z, ua, ub, old, tab_s, H);
                    } else {
                        nw = ising_decide8<RULE>(A, H - 16 - pr.y, ua, ub, old, tab_s, H);
                    }
                    if (nw != old) {
                        sp[k] = nw;
                        nflip += __popc((nw ^ old) & live);
                    }
                    i = inext;
                    pr = prn;
                    nc = ncn;
#pragma unroll
                    for (int q = 0; q < 4; ++q) e4[q] = e4n[q];
                }
                if (lev + 1 < L) {   // the next level's first position (clamped, see above)
                    const int32_t i2 = min(end + li, n - 1);
                    pr = pos[i2];
                    const uint32_t *ep = nib_ell_row(es, i2, W);
#pragma unroll
                    for (int q = 0; q < 4; ++q) e4[q] = ep[q * 32];
                    if constexpr (BIASED) nc = d.nibc[pr.x & 0xFFFFFF];
                }
                nib_barrier(1 + gl, tpg, gpc);
            }
        }
        // spins that changed at a visit, summed per warp into the controller
        unsigned long long v = nflip;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0ull)
            atomicAdd(reinterpret_cast<unsigned long long *>(&const_cast<DevCtl *>(ctl)->sweep_flips), v);

        // energy from the definition E = -1/2 sum_k s_k h_k over the last
        // sweep's ELL rows (|s h| <= 30 per vertex: int32 per thread), and the
        // write-back of the eight rows
        int32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const size_t sb = (size_t)slot * S + (S - 1);   // S >= 1 (sweep_nibble_ok)
        const uint32_t *es = d.sell + sb * ell_stride;
        const int2 *pos = d.spos + sb * (size_t)n;
        for (int32_t i = li; i < n; i += tpg) {
            const int2 p0 = pos[i];
            const uint32_t *ep = nib_ell_row(es, i, W);
            const uint32_t w = sp[p0.x & 0xFFFFFF];
            if constexpr (BIASED) {
                const int4 c = d.nibc[p0.x & 0xFFFFFF];
                uint32_t A = (uint32_t)c.x, A2 = (uint32_t)c.y;
                for (int q = 0; q < W; ++q) {
                    const uint32_t e = ep[q * 32];
                    const uint32_t v = sp[e & 0xFFFFFFu] * (uint32_t)((int32_t)e >> 24);
                    if (q < 8) A += v;
                    else A2 += v;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int32_t nq = (int32_t)((A >> (4 * q)) & 0xFu) + (int32_t)((A2 >> (4 * q)) & 0xFu);
                    const int32_t h = 2 * nq + c.z - H;   // c.z = H - sum_j |J_kj|
                    acc[q] += ((w >> (4 * q)) & 1u) ? h : -h;
                }
            } else {
                uint32_t A = 0x88888888u;
#pragma unroll
                for (int q = 0; q < W; ++q) {
                    const uint32_t e = ep[q * 32];
                    A += sp[e & 0xFFFFFFu] * (uint32_t)((int32_t)e >> 24);
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int32_t h = 2 * ((int32_t)((A >> (4 * q)) & 0xFu) - 8) - p0.y;   // p0.y = sum_j J_kj
                    acc[q] += ((w >> (4 * q)) & 1u) ? h : -h;
                }
            }
        }
        for (int32_t k = li; k < n; k += tpg) {
            const uint32_t w = sp[k];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (r0 + q < R) dst[(size_t)(r0 + q) * n + k] = ((w >> (4 * q)) & 1u) ? 1 : -1;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            long long v2 = acc[q];
            for (int o = 16; o > 0; o >>= 1) v2 += __shfl_down_sync(0xffffffffu, v2, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&red[gl * 8 + q], (unsigned long long)v2);
        }
    }
    __syncthreads();
    if (active && li < 8 && r0 + li < R) E_dst[r0 + li] = -((long long)red[gl * 8 + li] / 2);
}

template <int RULE, int WC, bool BIASED>
__global__ void __launch_bounds__(1024) k_sweep_ising_nib(SweepDesc d, int gpc, int tpg) {
    nib_body<RULE, WC, BIASED>(d, NibKeys{d.K}, d.t, d.slot, d.src, d.dst, d.E_dst, gpc, tpg, blockIdx.x);
}

// Many instances in one launch: CTA b works on member items[b].x, its block
// of groups items[b].y; the step index comes from the member's controller.
template <int RULE, bool BIASED>
__global__ void __launch_bounds__(1024)
k_sweep_ising_nib_batched(const SweepDesc *__restrict__ descs, const int2 *__restrict__ items, int gpc, int tpg) {
    const int2 it = items[blockIdx.x];
    const SweepDesc &d = descs[it.x];
    const int32_t t = d.ctl->t;
    if (t >= d.t_end) return;
    nib_body<RULE, 0, BIASED>(d, NibKeysSeed{d.K.k0[0], d.K.k1[0]}, t, t % d.slots, d.sp[t & 1],
                              d.sp[(t + 1) & 1], d.en[(t + 1) & 1], gpc, tpg, it.y);
}

}  // namespace

bool sweep_nibble_enabled() {
    const char *env = getenv("PAMC_SWEEP_NIBBLE");
    return !(env && env[0] == '0');
}

bool sweep_nibble_ok(int32_t H, int32_t S, int32_t ell_w, int lanes_per_vertex, bool global_spins,
                     bool biased_ok) {
    const bool fixed = H <= kNibbleMaxH && (ell_w == 4 || ell_w == 8);
    return (fixed || biased_ok) && S > 0 && lanes_per_vertex == 1 && !global_spins && sweep_nibble_enabled();
}

bool nibble_biased_constants(int32_t n, const int32_t *rp, const uint32_t *adj, int32_t H, int32_t ell_w,
                             std::vector<int4> &out) {
    if (!(ell_w == 4 || ell_w == 8 || ell_w == 12 || ell_w == 16) || H > kNibbleBiasedMaxH) return false;
    out.assign((size_t)n, make_int4(0, 0, 0, 0));
    for (int32_t k = 0; k < n; ++k) {
        int32_t slot = 0, half[2] = {0, 0}, neg[2] = {0, 0};
        for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
            const int32_t J = (int32_t)adj[e] >> 24;
            if (J == 0) continue;   // the ELL rows hold the nonzero couplings only
            const int hf = slot < 8 ? 0 : 1;
            half[hf] += J < 0 ? -J : J;
            neg[hf] += J < 0 ? -J : 0;
            ++slot;
        }
        if (slot > ell_w || half[0] > kNibbleHalfMaxH || half[1] > kNibbleHalfMaxH) return false;
        out[k] = make_int4((int32_t)((uint32_t)neg[0] * 0x11111111u), (int32_t)((uint32_t)neg[1] * 0x11111111u),
                           H - half[0] - half[1], 0);
    }
    return true;
}

size_t sweep_nibble_smem_bytes(int32_t n, int32_t H, SweepCfg cfg) {
    const int32_t n_pad = (n + 3) & ~3;
    return (((size_t)(2 * H + 1) * 8 + 15) & ~(size_t)15) + (size_t)cfg.groups_per_cta * n_pad * 4 +
           (size_t)cfg.groups_per_cta * 8 * 8;
}

cudaError_t launch_sweep_ising_nib(int rule, int32_t n, int32_t H, const pamc_params &p, int32_t t, int32_t slot,
                                   SchedView sv, const uint64_t *tab, const int8_t *src, const int32_t *parent,
                                   const int8_t *ncm_buf, const int32_t *ncm_idx, int8_t *dst, int64_t *E_dst,
                                   const DevCtl *ctl, SweepCfg cfg, cudaStream_t st, int32_t rbase) {
    const bool biased = sv.nibc != nullptr;
    if (!(sv.ell != nullptr && p.sweeps > 0 &&
          (biased ? (sv.W % 4 == 0 && sv.W >= 4 && sv.W <= 16 && H <= kNibbleBiasedMaxH)
                  : ((sv.W == 4 || sv.W == 8) && H <= kNibbleMaxH))))
        return cudaErrorInvalidValue;
    const int32_t groups = (p.R + 7) / 8;
    const int gpc = cfg.groups_per_cta, tpg = cfg.warps_per_group * 32;
    SweepDesc d;
    memset(&d, 0, sizeof(d));
    d.sorder = sv.order; d.slvl = sv.lvl_ptr; d.snlev = sv.nlev; d.sell = sv.ell; d.spos = sv.pos;
    d.tab = tab; d.src = src; d.parent = parent; d.ncm_buf = ncm_buf; d.ncm_idx = ncm_idx;
    d.dst = dst; d.E_dst = E_dst; d.ctl = ctl; d.n = n; d.n_pad = (n + 3) & ~3; d.H = H; d.R = p.R;
    d.S = p.sweeps; d.t = t; d.slot = slot; d.W = sv.W; d.K = make_philox_keys(p.seed);
    d.gbase = rbase / 4;
    d.nibc = sv.nibc;
    const size_t smem = sweep_nibble_smem_bytes(n, H, cfg);
    const int grid = (groups + gpc - 1) / gpc;
    cudaError_t err = cudaSuccess;
#define PAMC_NIB(RU, WV, BI)                                                                 \
    do {                                                                                     \
        err = allow_dynamic_smem(k_sweep_ising_nib<RU, WV, BI>, smem);                       \
        if (err != cudaSuccess) return err;                                                  \
        k_sweep_ising_nib<RU, WV, BI><<<grid, gpc * tpg, smem, st>>>(d, gpc, tpg);           \
    } while (0)
#define PAMC_NIB_W(RU)                                                                       \
    do {                                                                                     \
        if (!biased) {                                                                       \
            if (sv.W == 4) PAMC_NIB(RU, 4, false);                                           \
            else PAMC_NIB(RU, 8, false);                                                     \
        } else if (sv.W == 4) PAMC_NIB(RU, 4, true);                                         \
        else if (sv.W == 8) PAMC_NIB(RU, 8, true);                                           \
        else if (sv.W == 12) PAMC_NIB(RU, 12, true);                                         \
        else PAMC_NIB(RU, 16, true);                                                         \
    } while (0)
    if (rule == 0) PAMC_NIB_W(0);
    else PAMC_NIB_W(1);
#undef PAMC_NIB_W
#undef PAMC_NIB
    return cudaGetLastError();
}

cudaError_t launch_sweep_ising_nib_batched(int rule, bool biased, const SweepDesc *descs, const int2 *items,
                                           int32_t nitems, int32_t n_max, SweepCfg cfg, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    const int gpc = cfg.groups_per_cta, tpg = cfg.warps_per_group * 32;
    const size_t smem = sweep_nibble_smem_bytes(n_max, biased ? kNibbleBiasedMaxH : kNibbleMaxH, cfg);
    cudaError_t err;
#define PAMC_NIBB(RU, BI)                                                                    \
    do {                                                                                     \
        err = allow_dynamic_smem(k_sweep_ising_nib_batched<RU, BI>, smem);                   \
        if (err != cudaSuccess) return err;                                                  \
        k_sweep_ising_nib_batched<RU, BI><<<nitems, gpc * tpg, smem, st>>>(descs, items, gpc, tpg); \
    } while (0)
    if (rule == 0) {
        if (biased) PAMC_NIBB(0, true);
        else PAMC_NIBB(0, false);
    } else {
        if (biased) PAMC_NIBB(1, true);
        else PAMC_NIBB(1, false);
    }
#undef PAMC_NIBB
    return cudaGetLastError();
}

}  // namespace pamc
