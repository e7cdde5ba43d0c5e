// dense.cu -- the fully connected instance: J is an N x N int8 matrix in HBM
// (symmetric, +-1 off the diagonal, 0 on it).  Per temperature step:
//   k_dense_perm       the shared random order of each sweep (Sec. III.A):
//                      vertices sorted by (Philox key, index) -- bucket by the
//                      top key bits, then sort each bucket;
//   k_dense_tables     heat-bath T(h) (Eq. 4) or Metropolis T_M(2x) over the
//                      field range that does not saturate;
//   k_dense_recompute  H = J * S for the resampled population with
//                      mma.sync on e4m3 couplings (exact integer fields):
//                      the full recompute of every step when n is not a
//                      multiple of 16 (dense_tc.cu has the tcgen05 one);
//   k_dense_sweep      S sequential sweeps (cooperative, persistent): most
//                      CTAs own a slice of H rows (in tensor memory with the
//                      tcgen05 update, else in shared memory) and apply each
//                      block's flips (each flipped row of J read once for all
//                      replicas), a few CTAs run the per-replica decision
//                      chains of each block of kB positions.
#include <cooperative_groups.h>

#include "pamc_device.cuh"
#include "pamc_internal.h"
#include "tc_sm100.cuh"

namespace pamc {

namespace {

// ------------------------------------------------------------------ order
constexpr int kPermThreads = 1024;
constexpr int kPermBucketBits = 11;   // 2048 buckets

// The order of each sweep by (Philox key, index) in two launches.  Bucketing
// (one CTA per sweep): keys, a histogram over the top 11 key bits, a
// block-wide exclusive scan and a scatter into buckets (order within a bucket
// arbitrary).  Sorting (32 buckets per CTA): each bucket is ranked in shared
// memory by (key, index), which is unique, so the result is the exact order.
__global__ void __launch_bounds__(kPermThreads)
k_dense_perm_bucket(int32_t n, uint32_t key0, uint32_t key1, int32_t t, uint32_t *__restrict__ skey,
                    int32_t *__restrict__ sidx, int32_t *__restrict__ boff, const DevCtl *__restrict__ ctl) {
    constexpr int NB = 1 << kPermBucketBits;
    __shared__ int32_t cnt[NB];
    __shared__ int32_t wsum[kPermThreads / 32];
    if (ctl->done) return;
    const int32_t sw = blockIdx.x;
    uint32_t *kk = skey + (size_t)sw * n;
    int32_t *ii = sidx + (size_t)sw * n;
    int32_t *bo = boff + (size_t)sw * (NB + 1);
    for (int b = threadIdx.x; b < NB; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        const uint32_t key = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t, kTagPerm << 24, key0, key1).x;
        atomicAdd(&cnt[key >> (32 - kPermBucketBits)], 1);
    }
    __syncthreads();
    // exclusive scan of the NB counts: NB / blockDim consecutive buckets per thread
    constexpr int per = NB / kPermThreads;
    int32_t local[per], tot = 0;
#pragma unroll
    for (int i = 0; i < per; ++i) { local[i] = cnt[threadIdx.x * per + i]; tot += local[i]; }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t v = lane < kPermThreads / 32 ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < kPermThreads / 32) wsum[lane] = v;
    }
    __syncthreads();
    int32_t run = (x - tot) + (wid > 0 ? wsum[wid - 1] : 0);
#pragma unroll
    for (int i = 0; i < per; ++i) {
        const int b = threadIdx.x * per + i;
        bo[b] = run;
        cnt[b] = run;
        run += local[i];
    }
    if (threadIdx.x == 0) bo[NB] = n;
    __syncthreads();
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        const uint32_t key = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t, kTagPerm << 24, key0, key1).x;
        const int32_t p = atomicAdd(&cnt[key >> (32 - kPermBucketBits)], 1);
        kk[p] = key;
        ii[p] = k;
    }
}

constexpr int kSortBuckets = 32;        // buckets per sorting CTA
constexpr int kSortCap = 6144;          // items staged in shared memory (larger ranges sort in place)

__device__ __forceinline__ bool perm_before(uint32_t ka, int32_t ia, uint32_t kb, int32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

__global__ void __launch_bounds__(256)
k_dense_perm_sort(int32_t n, const uint32_t *__restrict__ skey, const int32_t *__restrict__ sidx,
                  const int32_t *__restrict__ boff, int32_t *__restrict__ perm, const DevCtl *__restrict__ ctl) {
    constexpr int NB = 1 << kPermBucketBits;
    __shared__ uint32_t ks[kSortCap];
    __shared__ int32_t is[kSortCap];
    if (ctl->done) return;
    const int32_t sw = blockIdx.y;
    const uint32_t *kk = skey + (size_t)sw * n;
    const int32_t *ii = sidx + (size_t)sw * n;
    const int32_t *bo = boff + (size_t)sw * (NB + 1);
    int32_t *out = perm + (size_t)sw * n;
    const int b0 = blockIdx.x * kSortBuckets;
    const int32_t lo = bo[b0], hi = bo[b0 + kSortBuckets];
    const bool staged = hi - lo <= kSortCap;
    if (staged)
        for (int32_t x = lo + threadIdx.x; x < hi; x += blockDim.x) { ks[x - lo] = kk[x]; is[x - lo] = ii[x]; }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = b0 + warp; b < b0 + kSortBuckets; b += blockDim.x / 32) {
        const int32_t blo = bo[b], bhi = bo[b + 1];
        for (int32_t xi = blo + lane; xi < bhi; xi += 32) {
            const uint32_t kx = staged ? ks[xi - lo] : kk[xi];
            const int32_t ix = staged ? is[xi - lo] : ii[xi];
            int32_t rank = 0;
            for (int32_t y = blo; y < bhi; ++y) {
                const uint32_t ky = staged ? ks[y - lo] : kk[y];
                const int32_t iy = staged ? is[y - lo] : ii[y];
                rank += perm_before(ky, iy, kx, ix) ? 1 : 0;
            }
            out[blo + rank] = ix;
        }
    }
}

// ------------------------------------------------------------------ tables
// Heat-bath: tab[i] = T(i - Hc), i in [0, 2Hc]; Metropolis: tab[x] = T_M(2x),
// x in [0, Hc].  When Hc < n the table must reach saturation at its ends
// (T(Hc) = 2^32, T(-Hc) = 0; T_M(2Hc) = 0), else PAMC_ERR_RANGE.
__global__ void k_dense_tables(int rule, int32_t Hc, int32_t n, DevCtl *__restrict__ ctl,
                               uint64_t *__restrict__ tab) {
    if (ctl->done) return;
    const double beta = ctl->beta;
    const int32_t cntv = rule == 0 ? 2 * Hc + 1 : Hc + 1;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cntv; i += gridDim.x * blockDim.x) {
        uint64_t v;
        if (rule == 0) v = thr_heatbath(beta, (int64_t)(i - Hc));
        else v = thr_metropolis(beta, 2 * (int64_t)i);
        tab[i] = v;
        if (Hc < n) {
            if (rule == 0 && i == 0 && v != 0) atomicCAS(&ctl->err, 0, (int)PAMC_ERR_RANGE);
            if (rule == 0 && i == 2 * Hc && v != (1ull << 32)) atomicCAS(&ctl->err, 0, (int)PAMC_ERR_RANGE);
            if (rule == 1 && i == Hc && v != 0) atomicCAS(&ctl->err, 0, (int)PAMC_ERR_RANGE);
        }
    }
}

// ------------------------------------------------------------------ recompute
// H[r][j] = sum_k J[j][k] S[r][k] with mma.m16n8k32 e4m3 x e4m3 -> f32.  J is
// stored in HBM as e4m3 bytes (+-1 and 0 are exact), the spins are converted
// to e4m3 while staged.  Every product is +-1 or 0 and every partial sum an
// integer of magnitude < 2^24, so the f32 result is the exact integer field
// (a GPU test sets a replica equal to a row of J, |h| = n - 1 up to 99,999,
// and compares every field with an exact product).
// A = J (row-major, K contiguous), B = S^T (column-major: each replica's spin
// row is K-contiguous).  One CTA per row slice of kRcRows rows and all
// (<= 64) replicas; K streamed through shared memory with cp.async.
constexpr int kRcWarps = 21;                  // 2 m16 tiles per warp
constexpr int kRcRows = kRcWarps * 32;        // 672 rows per CTA
constexpr int kRcK = 64;                      // K bytes per stage
constexpr int kRcStages = 3;                  // stages in flight
constexpr int kRcAStride = kRcK + 16;         // padded row stride (bank spread)
constexpr int kRcStageBytes = kRcRows * kRcAStride + 64 * kRcAStride;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;\n" ::); }

// +-1 int8 spins -> e4m3 (+1.0 = 0x38, -1.0 = 0xB8), four at a time
__device__ __forceinline__ uint32_t spins_to_e4m3(uint32_t x) { return (x & 0x80808080u) | 0x38383838u; }

// e4m3 coupling byte (0x38, 0xB8 or 0) -> +1, -1, 0
__device__ __forceinline__ int32_t e4m3_pm1(uint32_t b) {
    return ((int32_t)(int8_t)(uint8_t)b >> 7) | (int32_t)(b != 0u);
}

// stage kc of J rows and e4m3 spins into shared stage buffer `stage`
__device__ __forceinline__ void rc_load_stage(uint8_t *sm, const uint8_t *__restrict__ J,
                                              const int8_t *const *rowp, int32_t n, int32_t row0,
                                              int32_t kc, int stage) {
        uint8_t *As = sm + (size_t)stage * kRcStageBytes;
        uint8_t *Bs = As + (size_t)kRcRows * kRcAStride;
        const int32_t k0 = kc * kRcK;
        // each 16-byte piece is either copied asynchronously (aligned, in
        // range) or written synchronously -- never both
        for (int x = threadIdx.x; x < kRcRows * (kRcK / 16); x += blockDim.x) {
            const int rr = x / (kRcK / 16), cc = (x % (kRcK / 16)) * 16;
            const int32_t row = row0 + rr, col = k0 + cc;
            uint8_t *d = As + rr * kRcAStride + cc;
            if ((n & 15) == 0 && row < n && col + 16 <= n) {
                cp_async16(d, J + (size_t)row * n + col);
            } else {
                for (int q = 0; q < 16; ++q)
                    d[q] = (row < n && col + q < n) ? J[(size_t)row * n + col + q] : (uint8_t)0;
            }
        }
        for (int x = threadIdx.x; x < 64 * (kRcK / 16); x += blockDim.x) {
            const int rr = x / (kRcK / 16), cc = (x % (kRcK / 16)) * 16;
            const int32_t col = k0 + cc;
            const int8_t *p = rowp[rr];
            uint8_t *d = Bs + rr * kRcAStride + cc;
            // raw +-1 spins, converted to e4m3 when the fragments are read;
            // padding is harmless (J is zero there or the replica is unused)
            if (p != nullptr && col + 16 <= n && (((uintptr_t)(p + col)) & 15) == 0) {
                cp_async16(d, p + col);
            } else {
                for (int q = 0; q < 16; ++q) d[q] = (p != nullptr && col + q < n) ? (uint8_t)p[col + q] : (uint8_t)1;
            }
        }
        cp_async_commit();
    }

__global__ void __launch_bounds__(kRcWarps * 32, 1)
k_dense_recompute(int32_t n, int32_t R, const uint8_t *__restrict__ J, const int8_t *__restrict__ src,
                  const int32_t *__restrict__ parent, const int8_t *__restrict__ ncm_buf,
                  const int32_t *__restrict__ ncm_idx, int32_t *__restrict__ H,
                  const DevCtl *__restrict__ ctl, int restart_t) {
    extern __shared__ __align__(16) uint8_t sm[];
    // restart_t >= 0: only in the iteration whose controller restarted
    if (restart_t >= 0 ? !(ctl->restart && ctl->t == restart_t) : ctl->done != 0) return;
    const int32_t row0 = blockIdx.x * kRcRows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tig = lane & 3;
    __shared__ const int8_t *rowp[64];
    if (threadIdx.x < 64) {
        const int r = threadIdx.x;
        const int8_t *p = nullptr;
        if (r < R) {
            const int32_t q = ncm_idx[r];
            p = q >= 0 ? ncm_buf + (size_t)q * n : src + (size_t)parent[r] * n;
        }
        rowp[r] = p;
    }
    __syncthreads();
    float acc[2][8][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

    const int32_t nk = (n + kRcK - 1) / kRcK;
    for (int st = 0; st < kRcStages - 1; ++st) {
        if (st < nk) rc_load_stage(sm, J, rowp, n, row0, st, st);
        else cp_async_commit();
    }
    for (int32_t kc = 0; kc < nk; ++kc) {
        // keep kRcStages-1 stages in flight
        if (kc + kRcStages - 1 < nk)
            rc_load_stage(sm, J, rowp, n, row0, kc + kRcStages - 1, (kc + kRcStages - 1) % kRcStages);
        else
            cp_async_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kRcStages - 1));
        __syncthreads();
        const uint8_t *As = sm + (size_t)(kc % kRcStages) * kRcStageBytes;
        const uint8_t *Bs = As + (size_t)kRcRows * kRcAStride;
#pragma unroll
        for (int ks = 0; ks < kRcK; ks += 32) {
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const uint8_t *ar = As + (size_t)(warp * 32 + mt * 16 + g) * kRcAStride + ks + tig * 4;
                a[mt][0] = *reinterpret_cast<const uint32_t *>(ar);
                a[mt][1] = *reinterpret_cast<const uint32_t *>(ar + 8 * kRcAStride);
                a[mt][2] = *reinterpret_cast<const uint32_t *>(ar + 16);
                a[mt][3] = *reinterpret_cast<const uint32_t *>(ar + 8 * kRcAStride + 16);
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint8_t *br = Bs + (size_t)(nt * 8 + g) * kRcAStride + ks + tig * 4;
                const uint32_t b0 = spins_to_e4m3(*reinterpret_cast<const uint32_t *>(br));
                const uint32_t b1 = spins_to_e4m3(*reinterpret_cast<const uint32_t *>(br + 16));
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    asm volatile(
                        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]),
                          "+f"(acc[mt][nt][3])
                        : "r"(a[mt][0]), "r"(a[mt][1]), "r"(a[mt][2]), "r"(a[mt][3]), "r"(b0), "r"(b1));
                }
            }
        }
        __syncthreads();
    }
    cp_async_wait_all();
    // C fragment: rows g / g+8, columns (replicas) 2*tig, 2*tig+1
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int32_t row = row0 + warp * 32 + mt * 16 + g + (c >= 2 ? 8 : 0);
                const int r = nt * 8 + tig * 2 + (c & 1);
                if (row < n && r < R) H[(size_t)r * n + row] = __float2int_rn(acc[mt][nt][c]);
            }
}

// ------------------------------------------------------------------ sweep
constexpr int kSwThreads = 768;
constexpr int kB = 256;              // positions per block
constexpr int kC = kB / 32;          // positions per lane in a chain warp
// Chain tiles hold one bit per coupling (+1 set; J is +-1 off the diagonal):
// row m is kC words, bit l of word c for column position 32 c + l
// A chain applies the row of a flipped position m of its own block to the
// positions after m only (the earlier ones are decided), so of the tile
// J[P_q][P_q] only the words holding some column > m are produced: row m
// needs words floor((m + 1) / 32) .. kC - 1.  Rows with the same k =
// floor((m + 1) / 32) form a segment: rows 0..30 for k = 0, rows 32k-1 ..
// 32k+30 for k >= 1, each with kC - k words.
constexpr int tile_words_upper() {
    int w = 31 * kC;
    for (int k = 1; k < kC; ++k) w += 32 * (kC - k);
    return w;
}
constexpr int kTileWordsT = tile_words_upper();
constexpr int kTileWords = kTileWordsT + kB * kC;   // both tiles of a block
// When few positions flip (late in an anneal most blocks have a handful),
// the tile J[P_{q-1}][P_q] is not produced by the update CTAs: each chain CTA
// loads the rows of the positions its own replicas flipped in block q-1 at the
// end of that block's chain.  The update CTAs decide per block from the count
// of flipped positions two blocks earlier (the same count in every CTA).
constexpr int kT2Rare = 16;
// ... and in those blocks the row of a flip is staged while the chain runs:
// the first replica of a group to flip a position copies the row's 4-byte
// pieces that hold the next block's columns into a staging slot
constexpr int kStgSlots = 32;
// word wd of a block's production list -> tile (0: J[P_q][P_q], 1:
// J[P_{q-1}][P_q]) and word index m * kC + c within it
__device__ __forceinline__ void tile_word(int32_t wd, int &which, int32_t &ee) {
    if (wd >= kTileWordsT) {
        which = 1;
        ee = wd - kTileWordsT;
        return;
    }
    which = 0;
    int32_t base = 0;
    int k = 0;
    for (; k < kC - 1; ++k) {
        const int32_t words = (k == 0 ? 31 : 32) * (kC - k);
        if (wd < base + words) break;
        base += words;
    }
    const int32_t local = wd - base;
    const int32_t m = (k == 0 ? 0 : 32 * k - 1) + local / (kC - k);
    ee = m * kC + k + local % (kC - k);
}
constexpr int kWin = 4096;           // threshold entries kept in shared memory
constexpr long long kBarCycles = 4000000000ll;   // ~2 s: a barrier wait gives up after this

// tensor-core field update (TCU): the update CTA's fields live in tensor
// memory, one 128-row tile of 64 replica columns per 128 rows; a block's flips
// are applied as H += J[flipped, slice]^T D with D = +-2 (the new spin) or 0
constexpr int kTuTileBytes = 128 * 128;       // one K slice of one A tile
constexpr int kTuMaxTiles = 6;                // <= 768 rows per update CTA
constexpr int kTuBSlice = 64 * 128;           // one K slice of B (64 replicas)
constexpr uint32_t kTuCols = 512;             // tensor memory columns allocated
constexpr uint32_t kTuIdesc = (1u << 4) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// A rows of a 128-row tile are permuted so that the transposed 32-bit shared
// stores of a warp hit 32 distinct banks: A row 128b + 8s + g <-> slice row
// 128b + 16g + s (g < 8, s < 16)
__device__ __forceinline__ int32_t tu_row_of(int32_t arow) {
    return (arow & ~127) + ((arow & 7) << 4) + ((arow >> 3) & 15);
}
__device__ __forceinline__ int32_t tu_arow_of(int32_t row) {
    return (row & ~127) + ((row & 15) << 3) + ((row >> 4) & 7);
}
// byte offset of (row a of an A tile or replica row of B, k) in a 128-byte-
// swizzled K-major slice
__device__ __forceinline__ uint32_t tu_sw_off(int32_t row, int32_t kk) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((kk >> 4) ^ row) & 7) << 4) + (kk & 15));
}

struct GridBar {
    unsigned int count;
    unsigned int gen;
    int32_t t2_mode[4];   // block b's tile J[P_{b-1}][P_b] produced by the update CTAs (slot b % 4)
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch: one monotonic arrival counter;
// phase g completes when it reaches (g + 1) * nblocks.  Split in two so that
// a CTA can issue independent memory work between its arrival and its wait.
// The wait is bounded by the clock: after kBarCycles it sets
// PAMC_ERR_TIMEOUT and the kernel returns.
__device__ void grid_arrive(GridBar *bar) {
    __syncthreads();
    // the release add publishes the CTA's writes (ordered before it by the
    // CTA barrier); the acquire load that sees the last arrival makes every
    // CTA's writes visible to this one
    if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->count) : "memory");
}

__device__ bool grid_wait(GridBar *bar, unsigned int nblocks, unsigned int &gen, DevCtl *ctl, int *s_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int target = (gen + 1u) * nblocks;
        const long long start = clock64();
        int spins = 0;
        while ((int)(ld_acquire_u32(&bar->count) - target) < 0) {
            if (++spins > 256) {
                __nanosleep(20);
                if (clock64() - start > kBarCycles) {
                    atomicCAS(&ctl->err, 0, (int)PAMC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        gen += 1;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ bool grid_barrier(GridBar *bar, unsigned int nblocks, unsigned int &gen, DevCtl *ctl, int *s_ok) {
    grid_arrive(bar);
    return grid_wait(bar, nblocks, gen, ctl, s_ok);
}

struct DenseSweepArgs {
    int32_t n, R, S, rule, Hc;
    int32_t n_upd;            // CTAs that own H rows (the others run chains)
    int32_t rows_per;         // rows per update CTA
    int32_t ntiles;           // tensor-core update: 128-row tiles per update CTA
    int32_t t;
    PhiloxKeys K;
    const uint8_t *J;         // e4m3 couplings
    const int32_t *perm;      // [S][n]
    const uint64_t *tab;
    const int8_t *src;        // previous population (resampling parents)
    const int32_t *parent;
    const int8_t *ncm_buf;
    const int32_t *ncm_idx;
    int32_t *H;               // [R][n] in: recomputed fields; out: fields after the sweeps
    int8_t *dst;              // [R][n]
    int64_t *E;               // [R]
    int32_t *G;               // [2][kB][64] published fields of a block
    uint32_t *T;              // [2][kB][kC] bit tile J[P_q][P_q]
    uint32_t *T2;             // [2][kB][kC] bit tile J[P_{q-1}][P_q]
    unsigned long long *flip; // [3][kB] replica bit masks of flips
    unsigned long long *snew; // [3][kB] replica bit masks of the new spin (+1)
    GridBar *bar;
    DevCtl *ctl;
    int32_t gbase;            // group index of the first local replica group in the whole population
};

__device__ __forceinline__ const int8_t *pop_row(const DenseSweepArgs &a, int r) {
    const int32_t qn = a.ncm_idx[r];
    return qn >= 0 ? a.ncm_buf + (size_t)qn * a.n : a.src + (size_t)a.parent[r] * a.n;
}

// The S sweeps of one step.  Block q (kB consecutive positions of a sweep's
// order) is decided by the chain CTAs in phase q while the update CTAs apply
// block q-1 to their rows; the fields a chain starts from were published in
// phase q-1 (all blocks up to q-2 applied) and the chain adds block q-1's
// flips itself from the tile J[P_{q-1}][P_q].  One grid barrier per block.
template <bool TCU>
__global__ void __launch_bounds__(kSwThreads, 1) k_dense_sweep(DenseSweepArgs a) {
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ int s_ok, s_nl;
    __shared__ int32_t s_wlo, s_wn;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    __shared__ int32_t s_nown, s_nu, s_nslot;
    if (a.ctl->done) return;
    const int32_t n = a.n, R = a.R;
    const unsigned int nblocks = gridDim.x;
    unsigned int gen = 0;
    const bool upd = (int)blockIdx.x < a.n_upd;
    const int32_t nb = (n + kB - 1) / kB;              // blocks per sweep
    const int32_t total = nb * a.S;                    // blocks of the step
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto block_pos = [&](int32_t q) { return a.perm + (size_t)(q / nb) * n + (size_t)(q % nb) * kB; };
    auto block_cnt = [&](int32_t q) { return min(kB, n - (q % nb) * kB); };

    // ---------------- update CTA shared memory
    const int32_t ua = upd ? blockIdx.x * a.rows_per : 0;
    const int32_t ub = upd ? max(ua, min(n, ua + a.rows_per)) : 0;
    const int32_t rows = ub - ua;
    const int32_t rw = (a.rows_per + 31) / 32;
    // TCU: [A: 2 K slices x ntiles tiles][B: 2 K slices] 1024-aligned, then the rest
    uint8_t *tu_base = sm + ((1024u - (smem_u32(sm) & 1023u)) & 1023u);
    uint8_t *tuA = tu_base;
    uint8_t *tuB = tuA + (size_t)2 * a.ntiles * kTuTileBytes;
    // 16-byte aligned, as dense_sweep_smem counts it (the 64-bit masks below need it)
    uint8_t *after = TCU ? tuB + 2 * kTuBSlice : sm + (((size_t)R * a.rows_per * 4 + 15) & ~(size_t)15);
    int32_t *Hs = reinterpret_cast<int32_t *>(sm);
    uint32_t *ubits = reinterpret_cast<uint32_t *>(after);
    unsigned long long *fprev = reinterpret_cast<unsigned long long *>(
        after + ((((size_t)R * rw * 4) + 15) & ~(size_t)15));
    unsigned long long *sprev = fprev + kB;
    int32_t *Pprev = reinterpret_cast<int32_t *>(sprev + kB);
    int32_t *Pring = Pprev + kB;                       // positions of block b in slot b % 4 (TCU)
    int32_t *Pcur = Pring;
    int32_t *Pnext = Pring + kB;
    int32_t *flist = Pring + 4 * kB;
    int32_t *ownl = flist + kB;                        // TCU: block positions owned by this CTA
    auto ring_slot = [&](int32_t b) { return Pring + (size_t)(b & 3) * kB; };
    // ---------------- chain CTA shared memory
    const int cg = blockIdx.x - a.n_upd;               // chain group (4 replicas)
    const int32_t nw = (n + 31) / 32;
    uint32_t *tile = reinterpret_cast<uint32_t *>(sm);             // J[P_q][P_q]
    uint32_t *tile2 = tile + (size_t)kB * kC;                      // J[P_{q-1}][P_q]
    uint32_t *cbits = tile2 + (size_t)kB * kC;
    uint64_t *win = reinterpret_cast<uint64_t *>(cbits + (((size_t)4 * nw + 3) & ~(size_t)3));
    int32_t *Gs = reinterpret_cast<int32_t *>(win + kWin);
    int32_t *thr_all = Gs + 4 * kB;                                 // [2][4][kB]: block b in b & 1
    int32_t *Pc = thr_all + 8 * kB;
    unsigned long long *cfm = reinterpret_cast<unsigned long long *>(Pc + kB);
    unsigned long long *csn = cfm + kB;
    uint32_t *udraw = reinterpret_cast<uint32_t *>(csn + kB);      // [4][kB] draws of a block
    uint32_t *gmask = udraw + 4 * kB;      // [kB] the group's replicas that flipped at a position
    int32_t *Ulist = reinterpret_cast<int32_t *>(gmask + kB);     // [kB] positions some of them flipped
    int32_t *Pnx = Ulist + kB;                                     // [kB] positions of the next block
    uint32_t *stg = reinterpret_cast<uint32_t *>(Pnx + kB);       // [kStgSlots][kC][32] staged row pieces
    int32_t *Uslot = reinterpret_cast<int32_t *>(stg + (size_t)kStgSlots * kC * 32);   // [kStgSlots] their positions
    // thresholds of block qb for the group's 4 replicas (Eq. 4 / Metropolis
    // inverted to field values) into thr_all[qb & 1], by nthr threads from
    // tid0 (all of the CTA, or a group of warps synchronised by named barrier
    // bar): one Philox call per position (its four words are the four
    // replicas' draws), then (position, replica) items two at a time, the two
    // binary searches run in step so that their table reads overlap.
    // Positions come from P.
    auto thresholds = [&](int32_t qb, const int32_t *P, int32_t tid0, int32_t nthr, int bar) {
        const int32_t cnt = block_cnt(qb);
        const int32_t sw = qb / nb;
        const bool inwin = s_wn <= kWin;
        const int32_t t = (int32_t)threadIdx.x - tid0;
        int32_t *thr = thr_all + (size_t)(qb & 1) * 4 * kB;
        for (int32_t m = t; m < cnt; m += nthr) {
            const u32x4 u = philox_rk((uint32_t)P[m], (uint32_t)sw, (uint32_t)a.t, (kTagFlip << 24) | (uint32_t)(cg + a.gbase), a.K);
            udraw[m] = u.x;
            udraw[kB + m] = u.y;
            udraw[2 * kB + m] = u.z;
            udraw[3 * kB + m] = u.w;
        }
        if (nthr == (int32_t)blockDim.x) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
        auto tv = [&](int32_t i) -> uint64_t { return inwin ? win[i] : a.tab[i]; };
        for (int32_t xa = t; xa < 4 * cnt; xa += 2 * nthr) {
            const int32_t xb = xa + nthr;
            const bool vb = xb < 4 * cnt;
            const int32_t ma = xa >> 2, mb = vb ? (xb >> 2) : ma;
            const uint64_t uqa = udraw[(xa & 3) * kB + ma], uqb = udraw[(xb & 3) * kB + mb];
            int32_t ra, rb;
            if (a.rule == 0) {
                // smallest h with T(h) > u: s = +1 iff h >= res
                const int32_t top = inwin ? s_wn - 1 : 2 * a.Hc + 1;
                int32_t loa = 0, hia = top, lob = 0, hib = vb ? top : 0;
                while (loa < hia || lob < hib) {
                    const int32_t mida = (loa + hia) >> 1, midb = (lob + hib) >> 1;
                    const uint64_t ta = loa < hia ? tv(mida) : 0ull, tb = lob < hib ? tv(midb) : 0ull;
                    if (loa < hia) { if (ta > uqa) hia = mida; else loa = mida + 1; }
                    if (lob < hib) { if (tb > uqb) hib = midb; else lob = midb + 1; }
                }
                ra = (inwin ? loa + s_wlo : loa) - a.Hc;
                rb = (inwin ? lob + s_wlo : lob) - a.Hc;
            } else {
                // largest x with T_M(2x) > u: flip iff s*h <= res
                const int32_t top = inwin ? s_wn - 1 : a.Hc;
                int32_t loa = 0, hia = top, lob = 0, hib = vb ? top : 0;
                while (loa < hia || lob < hib) {
                    const int32_t mida = (loa + hia + 1) >> 1, midb = (lob + hib + 1) >> 1;
                    const uint64_t ta = loa < hia ? tv(mida) : 0ull, tb = lob < hib ? tv(midb) : 0ull;
                    if (loa < hia) { if (ta > uqa) loa = mida; else hia = mida - 1; }
                    if (lob < hib) { if (tb > uqb) lob = midb; else hib = midb - 1; }
                }
                ra = (loa == a.Hc && a.Hc >= n) ? n + 1 : loa;
                rb = (lob == a.Hc && a.Hc >= n) ? n + 1 : lob;
            }
            thr[(xa & 3) * kB + ma] = ra;
            if (vb) thr[(xb & 3) * kB + mb] = rb;
        }
    };

    // update CTAs: publish the fields of block qn's positions they own, and
    // gather their share of the tiles J[P_qn][P_qn] and J[P_{qn-1}][P_qn]
    // update CTAs publish, for block qn: the fields of the positions they own
    // (publish_G) and their share of the tiles J[P_qn][P_qn] and
    // J[P_{qn-1}][P_qn] (publish_tiles); publish_lists stages the position lists
    auto publish_lists = [&](int32_t qn) {
        const int32_t *P = block_pos(qn);
        const int32_t cnt = block_cnt(qn);
        if (threadIdx.x == 0) s_nown = 0;
        if ((int)threadIdx.x < cnt) Pnext[threadIdx.x] = P[threadIdx.x];
        if (qn > 0 && (int)threadIdx.x < block_cnt(qn - 1)) Pcur[threadIdx.x] = block_pos(qn - 1)[threadIdx.x];
        __syncthreads();
        if constexpr (TCU) {
            if ((int)threadIdx.x < cnt) {
                const int32_t p = Pnext[threadIdx.x];
                if (p >= ua && p < ub) ownl[atomicAdd(&s_nown, 1)] = (int32_t)threadIdx.x;
            }
            __syncthreads();
        }
    };
    auto publish_G = [&](int32_t qn) {
        const int32_t cnt = block_cnt(qn);
        int32_t *Gq = a.G + (size_t)(qn & 1) * kB * 64;
        if constexpr (TCU) {
            // an owned position's fields are four loads of 16 columns from its
            // tensor-memory lane; the warps of a lane quarter (warp % 4) deal
            // those loads out among themselves in list order
            const int quarter = warp & 3, share = warp >> 2;
            constexpr int kShares = (kSwThreads / 32) / 4;
            const int32_t nown = s_nown;
            int dealt = 0;
            for (int32_t o = 0; o < nown; ++o) {
                const int32_t m = ownl[o];
                const int32_t ar = tu_arow_of(Pnext[m] - ua);
                if (((ar & 127) >> 5) != quarter) continue;
                const uint32_t tbase = s_tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((ar >> 7) * 64);
                for (int c0 = 0; c0 < 64; c0 += 16, ++dealt) {
                    if (dealt % kShares != share) continue;
                    uint32_t v[16];
                    tc_ld16(tbase + (uint32_t)c0, v);
                    if (lane == (ar & 31))
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < R) Gq[m * 64 + c0 + j] = __float2int_rn(__uint_as_float(v[j]));
                }
            }
        } else {
            for (int32_t x = threadIdx.x; x < cnt * R; x += blockDim.x) {
                const int32_t m = x / R, r = x % R;
                const int32_t p = Pnext[m];
                if (p >= ua && p < ub) Gq[m * 64 + r] = Hs[r * a.rows_per + (p - ua)];
            }
        }
    };
    auto publish_tiles = [&](int32_t qn) {
        const int32_t cnt = block_cnt(qn);
        const int32_t per = (kTileWords + a.n_upd - 1) / a.n_upd;
        const int32_t w0 = blockIdx.x * per, w1 = min(kTileWords, w0 + per);
        const int32_t cntp = qn > 0 ? block_cnt(qn - 1) : 0;
        for (int32_t wd = w0 + warp; wd < w1; wd += kSwThreads / 32) {   // warp-uniform
            int which;
            int32_t ee;
            tile_word(wd, which, ee);
            const int32_t m = ee / kC, m2 = (ee % kC) * 32 + lane;
            bool pos = false;
            if (which == 0) {
                if (m < cnt && m2 < cnt) pos = e4m3_pm1(a.J[(size_t)Pnext[m] * n + Pnext[m2]]) > 0;
            } else {
                if (m < cntp && m2 < cnt) pos = e4m3_pm1(a.J[(size_t)Pcur[m] * n + Pnext[m2]]) > 0;
            }
            const uint32_t word = __ballot_sync(0xffffffffu, pos);
            if (lane == 0) (which == 0 ? a.T : a.T2)[(size_t)(qn & 1) * kB * kC + ee] = word;
        }
    };

    // TCU: this CTA's share of the tiles of block q+2 is loaded between its
    // arrival at the grid barrier that ends phase q and its wait (a warp's
    // first two tile words held in registers as raw coupling bytes, one per
    // lane) and packed and stored in phase q+1.  The entries are single bytes
    // at scattered places of J: their misses occupy the load pipeline for a
    // while, which costs least there.
    uint32_t tvA = 0u, tvB = 0u;
    bool tokA = false, tokB = false;   // the lane's coupling lies inside the block
    int32_t teA = -1, teB = -1;        // warp-uniform word indices
    auto tile_src = [&](int32_t qn, int32_t wd) -> const uint8_t * {   // nullptr: outside the block
        const int32_t cnt = block_cnt(qn), cntc = block_cnt(qn - 1);
        const int32_t *Pn = ring_slot(qn), *Pc = ring_slot(qn - 1);
        int which;
        int32_t ee;
        tile_word(wd, which, ee);
        const int32_t m = ee / kC, m2 = (ee % kC) * 32 + lane;
        if (which == 0) return (m < cnt && m2 < cnt) ? a.J + (size_t)Pn[m] * n + Pn[m2] : nullptr;
        return (m < cntc && m2 < cnt) ? a.J + (size_t)Pc[m] * n + Pn[m2] : nullptr;
    };
    auto tile_word_store = [&](int32_t qn, int32_t wd, uint32_t raw) {
        const uint32_t word = __ballot_sync(0xffffffffu, e4m3_pm1(raw) > 0);
        int which;
        int32_t ee;
        tile_word(wd, which, ee);
        if (lane == 0) (which == 0 ? a.T : a.T2)[(size_t)(qn & 1) * kB * kC + ee] = word;
    };
    auto tile_issue = [&](int32_t qn, int32_t words) {
        teA = teB = -1;
        if (qn >= total) return;
        // warps 1..: warp 0 polls the grid barrier meanwhile
        if (warp == 0) return;
        const int32_t per = (words + a.n_upd - 1) / a.n_upd;
        const int32_t w0 = blockIdx.x * per, w1 = min(words, w0 + per);
        constexpr int kNW = kSwThreads / 32 - 1;
        const int32_t wa = w0 + warp - 1, wb = wa + kNW;
        // unconditional loads (from J[0][0] outside the block), so that nothing
        // waits for them before the next phase
        if (wa < w1) { teA = wa; const uint8_t *src = tile_src(qn, wa); tokA = src != nullptr; tvA = *(tokA ? src : a.J); }
        if (wb < w1) { teB = wb; const uint8_t *src = tile_src(qn, wb); tokB = src != nullptr; tvB = *(tokB ? src : a.J); }
        for (int32_t wd = wa + 2 * kNW; wd < w1; wd += kNW) {   // more than two words per warp: now
            const uint8_t *src = tile_src(qn, wd);
            tile_word_store(qn, wd, src ? (uint32_t)*src : 0u);
        }
    };
    auto tile_flush = [&](int32_t qn) {
        if (teA >= 0) tile_word_store(qn, teA, tokA ? tvA : 0u);
        if (teB >= 0) tile_word_store(qn, teB, tokB ? tvB : 0u);
    };
    // chain CTAs, blocks whose J[P_{q-1}][P_q] is not produced: the rows of
    // the positions in Ulist (block q-1, Pc) over block q's positions (Pnx),
    // packed straight into the shared tile.  Word wd is row Ulist[wd / kC],
    // columns 32 (wd % kC) .. +31.  A warp's first two words are loaded at the
    // end of block q-1's chain and packed at the start of block q's.
    auto chain_word_store = [&](int32_t wd, bool ok, uint32_t raw) {
        const uint32_t word = __ballot_sync(0xffffffffu, ok && e4m3_pm1(raw) > 0);
        if (lane == 0) tile2[(size_t)Ulist[wd / kC] * kC + wd % kC] = word;
    };
    auto chain_src = [&](int32_t wd, int32_t cnt1, bool &ok) -> const uint8_t * {
        const int32_t m2 = (wd % kC) * 32 + lane;
        ok = m2 < cnt1;
        return ok ? a.J + (size_t)Pc[Ulist[wd / kC]] * n + Pnx[m2] : a.J;
    };
    auto chain_t2_issue = [&](int32_t nu, int32_t cnt1) {
        constexpr int kNW = kSwThreads / 32;
        const int32_t words = nu * kC, wa = warp, wb = warp + kNW;
        teA = teB = -1;
        if (wa < words) { teA = wa; tvA = *chain_src(wa, cnt1, tokA); }
        if (wb < words) { teB = wb; tvB = *chain_src(wb, cnt1, tokB); }
        for (int32_t wd = wa + 2 * kNW; wd < words; wd += kNW) {   // more than two words per warp: now
            bool ok;
            const uint8_t *src = chain_src(wd, cnt1, ok);
            chain_word_store(wd, ok, *src);
        }
    };
    auto chain_t2_flush = [&]() {
        if (teA >= 0) chain_word_store(teA, tokA, tvA);
        if (teB >= 0) chain_word_store(teB, tokB, tvB);
        teA = teB = -1;
    };

    // ---------------- prologue
    if (upd) {
        if constexpr (TCU) {
            if (warp == 0) tc_alloc(&s_tmem, kTuCols);
            if (threadIdx.x == 0) {
                mbar_init(&s_mbar, 1);
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
            // A and B start as zeros (finite operands wherever a K step reads past the flips)
            for (int32_t x = threadIdx.x; x < (2 * a.ntiles * kTuTileBytes + 2 * kTuBSlice) / 16; x += blockDim.x)
                reinterpret_cast<uint4 *>(tuA)[x] = make_uint4(0u, 0u, 0u, 0u);
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            // fields into tensor memory: warp w covers lane quarter w % 4 of some (tile, 16 columns)
            const int quarter = warp & 3;
            for (int32_t pr = warp >> 2; pr < a.ntiles * 4; pr += (kSwThreads / 32) / 4) {
                const int tile = pr >> 2, c0 = (pr & 3) * 16;
                const int32_t ar = tile * 128 + quarter * 32 + lane;
                const int32_t j = tu_row_of(ar);
                uint32_t v[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int r = c0 + c;
                    const int32_t hv = (j < rows && r < R) ? a.H[(size_t)r * n + ua + j] : 0;
                    v[c] = __float_as_uint((float)hv);
                }
                tc_st16(s_tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tile * 64 + c0), v);
            }
            tc_wait_st();
        } else {
            for (int32_t x = threadIdx.x; x < R * rows; x += blockDim.x) {
                const int r = x / rows, j = x % rows;
                Hs[r * a.rows_per + j] = a.H[(size_t)r * n + ua + j];
            }
        }
        for (int32_t x = threadIdx.x; x < R * rw; x += blockDim.x) {
            const int r = x / rw, w = x % rw;
            const int8_t *row = pop_row(a, r) + ua;
            uint32_t bits = 0;
            for (int b = 0; b < 32; ++b) {
                const int32_t j = w * 32 + b;
                if (j < rows && row[j] > 0) bits |= 1u << b;
            }
            ubits[r * rw + w] = bits;
        }
        if constexpr (TCU) tc_fence_before();
        __syncthreads();
        if constexpr (TCU) tc_fence_after();
        if (total > 0) {
            if constexpr (TCU) {
                Pnext = ring_slot(0);
                Pcur = ring_slot(3);
                for (int32_t b = 1; b <= 2; ++b)
                    if (total > b && (int)threadIdx.x < block_cnt(b)) ring_slot(b)[threadIdx.x] = block_pos(b)[threadIdx.x];
            }
            publish_lists(0);
            publish_G(0);
            publish_tiles(0);
            if constexpr (TCU) {
                __syncthreads();   // ring slot 1 written
                tile_issue(1, kTileWords);
            }
        }
    } else {
        for (int32_t x = threadIdx.x; x < 4 * nw; x += blockDim.x) {
            const int qq = x / nw, w = x % nw;
            const int r = cg * 4 + qq;
            uint32_t bits = 0;
            if (r < R) {
                const int8_t *row = pop_row(a, r);
                const int32_t k0 = w * 32;
                if (k0 + 32 <= n && (((uintptr_t)(row + k0)) & 15) == 0) {
                    const uint4 v0 = *reinterpret_cast<const uint4 *>(row + k0);
                    const uint4 v1 = *reinterpret_cast<const uint4 *>(row + k0 + 16);
                    const uint32_t wv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            bits |= (((wv[i] >> (8 * b)) & 0x80u) ? 0u : 1u) << (4 * i + b);
                } else {
                    for (int b = 0; b < 32; ++b) {
                        const int32_t k = k0 + b;
                        if (k < n && row[k] > 0) bits |= 1u << b;
                    }
                }
            }
            cbits[x] = bits;
        }
        if (blockIdx.x == a.n_upd && threadIdx.x < kB) {
            for (int z = 0; z < 3; ++z) { a.flip[z * kB + threadIdx.x] = 0ull; a.snew[z * kB + threadIdx.x] = 0ull; }
        }
        if (blockIdx.x == a.n_upd && (int)threadIdx.x < R) a.E[threadIdx.x] = 0;
        if (threadIdx.x == 0) s_nslot = 0;
        // the part of the threshold table where it is neither 0 nor 2^32
        // (heat-bath) or above 0 (Metropolis)
        if (threadIdx.x == 0) {
            int32_t lo, hi;
            if (a.rule == 0) {
                int32_t l = 0, h2 = 2 * a.Hc + 1;
                while (l < h2) { const int32_t md = (l + h2) >> 1; if (a.tab[md] > 0ull) h2 = md; else l = md + 1; }
                lo = l;
                l = lo; h2 = 2 * a.Hc + 1;
                while (l < h2) { const int32_t md = (l + h2) >> 1; if (a.tab[md] == (1ull << 32)) h2 = md; else l = md + 1; }
                hi = min(l, 2 * a.Hc);
            } else {
                int32_t l = 0, h2 = a.Hc + 1;
                while (l < h2) { const int32_t md = (l + h2) >> 1; if (a.tab[md] == 0ull) h2 = md; else l = md + 1; }
                lo = 0;
                hi = min(l, a.Hc);
            }
            s_wlo = lo;
            s_wn = hi - lo + 1;
        }
        __syncthreads();
        if (s_wn <= kWin)
            for (int32_t i = threadIdx.x; i < s_wn; i += blockDim.x) win[i] = a.tab[s_wlo + i];
    }
    uint32_t mphase = 0;     // TCU: completed phases of s_mbar
    // chain CTAs stage 4-byte pieces of J (its base must be 4-byte aligned)
    const bool stage_ok = (reinterpret_cast<uintptr_t>(a.J) & 3) == 0;
    // chain CTAs: whether the current block's J[P_{q-1}][P_q] was produced,
    // read one phase ahead (block 1's is, by the prologue)
    int32_t t2_cur = 1;
    // chain CTAs: this thread's position of the next block, loaded a phase ahead
    int32_t pcn = (!upd && total > 0) ? block_pos(0)[min((int32_t)threadIdx.x, block_cnt(0) - 1)] : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.bar->t2_mode[1] = 1;   // block 1's tile: produced in the prologue
    bool alive = grid_barrier(a.bar, nblocks, gen, a.ctl, &s_ok);
    for (int32_t q = 0; alive && q <= total; ++q) {
        int32_t nl_q = 0;          // update CTAs: positions of block q-1 that flipped in some replica
        if (upd) {
            bool issued = false;   // TCU: MMAs of this phase in flight
            // the independent loads go first: block q-1's flip masks and (TCU)
            // the positions of block q+3 (unconditional, from a clamped index:
            // nothing waits for them here)
            unsigned long long fl_in = 0ull, sn_in = 0ull;
            if (q > 0 && (int)threadIdx.x < block_cnt(q - 1)) {
                fl_in = a.flip[((q - 1) % 3) * kB + threadIdx.x];
                sn_in = a.snew[((q - 1) % 3) * kB + threadIdx.x];
            }
            int32_t pn3 = -1;
            bool pn3_ok = false;
            if constexpr (TCU) {
                const int32_t q3 = min(q + 3, total - 1);
                pn3_ok = q + 3 < total && (int)threadIdx.x < block_cnt(q3);
                pn3 = block_pos(q3)[min((int32_t)threadIdx.x, block_cnt(q3) - 1)];
            }
            // ---- apply block q-1 to the owned rows
            if (q > 0) {
                const int32_t qp = q - 1;
                const int32_t *P = TCU ? ring_slot(qp) : block_pos(qp);
                const int32_t cntp = block_cnt(qp);
                if (threadIdx.x == 0) s_nl = 0;
                __syncthreads();
                if ((int)threadIdx.x < cntp) {
                    const int32_t m = threadIdx.x;
                    const unsigned long long f = fl_in;
                    const int32_t p = P[m];
                    fprev[m] = f;
                    sprev[m] = sn_in;
                    Pprev[m] = p;
                    if (f != 0ull) {
                        flist[atomicAdd(&s_nl, 1)] = m;
                        if (p >= ua && p < ub) {
                            const int32_t lj = p - ua;
                            unsigned long long ff = f;
                            while (ff) {
                                const int r = __ffsll((long long)ff) - 1;
                                ff &= ff - 1;
                                atomicXor(&ubits[r * rw + (lj >> 5)], 1u << (lj & 31));
                            }
                        }
                    }
                }
                __syncthreads();
                const int32_t nl = s_nl;
                nl_q = nl;
                if (blockIdx.x == 0 && threadIdx.x == 0) {   // the only writer
                    a.ctl->dense_rows += nl;
                    a.ctl->dense_positions += cntp;
                }
                if constexpr (TCU) {
                    if (nl > 0) {
                        // A: the flipped positions' coupling rows over this slice,
                        // transposed 4x4 bytes at a time into K-major tiles; k = list
                        // index.  A warp task is 16 positions x 128 rows: lane (pg, rg)
                        // loads 16 rows (16 bytes) of 4 positions; two tasks per
                        // iteration keep eight 16-byte loads of a lane in flight
                        constexpr int kNW = kSwThreads / 32;
                        const int32_t ntask = ((nl + 15) >> 4) * a.ntiles;
                        const int pg = lane >> 3, rg = lane & 7;
                        for (int32_t t0 = warp; t0 < ntask; t0 += 2 * kNW) {
                            uint4 w[2][4];
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const int32_t task = t0 + u * kNW;
                                const int32_t c16 = task / a.ntiles, rb = task % a.ntiles;
                                const int32_t j0 = rb * 128 + rg * 16;         // slice rows j0 .. j0+15
#pragma unroll
                                for (int c = 0; c < 4; ++c) {
                                    const int32_t i = c16 * 16 + pg * 4 + c;
                                    w[u][c] = make_uint4(0u, 0u, 0u, 0u);
                                    if (task < ntask && i < nl && j0 < rows)
                                        w[u][c] = __ldg(reinterpret_cast<const uint4 *>(
                                            a.J + (size_t)Pprev[flist[i]] * n + ua + j0));
                                }
                            }
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const int32_t task = t0 + u * kNW;
                                if (task >= ntask) break;
                                const int32_t c16 = task / a.ntiles, rb = task % a.ntiles;
                                const int32_t k = c16 * 16 + pg * 4;
                                uint8_t *Ak = tuA + (size_t)(k >> 7) * a.ntiles * kTuTileBytes + (size_t)rb * kTuTileBytes;
#pragma unroll
                                for (int s4 = 0; s4 < 4; ++s4) {
                                    const uint32_t x0 = s4 == 0 ? w[u][0].x : s4 == 1 ? w[u][0].y : s4 == 2 ? w[u][0].z : w[u][0].w;
                                    const uint32_t x1 = s4 == 0 ? w[u][1].x : s4 == 1 ? w[u][1].y : s4 == 2 ? w[u][1].z : w[u][1].w;
                                    const uint32_t x2 = s4 == 0 ? w[u][2].x : s4 == 1 ? w[u][2].y : s4 == 2 ? w[u][2].z : w[u][2].w;
                                    const uint32_t x3 = s4 == 0 ? w[u][3].x : s4 == 1 ? w[u][3].y : s4 == 2 ? w[u][3].z : w[u][3].w;
                                    const uint32_t lo01 = __byte_perm(x0, x1, 0x5140), hi01 = __byte_perm(x0, x1, 0x7362);
                                    const uint32_t lo23 = __byte_perm(x2, x3, 0x5140), hi23 = __byte_perm(x2, x3, 0x7362);
                                    const uint32_t o[4] = {__byte_perm(lo01, lo23, 0x5410), __byte_perm(lo01, lo23, 0x7632),
                                                           __byte_perm(hi01, hi23, 0x5410), __byte_perm(hi01, hi23, 0x7632)};
#pragma unroll
                                    for (int r = 0; r < 4; ++r) {
                                        const int32_t ar = (4 * s4 + r) * 8 + rg;   // = tu_arow_of(j0 + 4 s4 + r) & 127
                                        *reinterpret_cast<uint32_t *>(Ak + tu_sw_off(ar, k & 127)) = o[r];
                                    }
                                }
                            }
                        }
                        // B = D^T: replica r, k -> +2 (new spin +1) / -2 / 0 as e4m3
                        const int32_t nk4 = ((nl + 31) >> 5) * 8;        // 4-byte words per replica row
                        for (int32_t x = threadIdx.x; x < 64 * nk4; x += blockDim.x) {
                            const int r = x / nk4;
                            const int32_t k0 = (x % nk4) * 4;
                            uint32_t wv = 0u;
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int32_t i = k0 + c;
                                if (i < nl && r < R) {
                                    const int32_t m = flist[i];
                                    if ((fprev[m] >> r) & 1ull)
                                        wv |= (((sprev[m] >> r) & 1ull) ? 0x40u : 0xC0u) << (8 * c);
                                }
                            }
                            *reinterpret_cast<uint32_t *>(tuB + (size_t)(k0 >> 7) * kTuBSlice + tu_sw_off(r, k0 & 127)) = wv;
                        }
                        fence_async_smem();
                        __syncthreads();
                        if (threadIdx.x == 0) {
                            tc_fence_after();
                            const int32_t ks = (nl + 31) >> 5;
                            for (int tl = 0; tl < a.ntiles; ++tl)
                                for (int32_t kq = 0; kq < ks; ++kq) {
                                    const uint32_t aaddr = smem_u32(tuA + (size_t)(kq >> 2) * a.ntiles * kTuTileBytes +
                                                                    (size_t)tl * kTuTileBytes);
                                    const uint32_t baddr = smem_u32(tuB + (size_t)(kq >> 2) * kTuBSlice);
                                    tc_mma(s_tmem + (uint32_t)(tl * 64), sw128_desc(aaddr) + (uint64_t)(2 * (kq & 3)),
                                           sw128_desc(baddr) + (uint64_t)(2 * (kq & 3)), kTuIdesc, 1u);
                                }
                            tc_commit(&s_mbar);
                        }
                        __syncwarp();
                        issued = true;   // waited for after the independent tile gather below
                    }
                    __syncthreads();
                } else {
                const int32_t j = threadIdx.x;
                const uint8_t *Jc = a.J + ua + j;
                for (int32_t base = 0; base < nl; base += 16) {
                    int32_t jv[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        jv[u] = (base + u < nl && j < rows) ? e4m3_pm1(Jc[(size_t)Pprev[flist[base + u]] * n]) : 0;
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        if (base + u >= nl) break;
                        const int32_t m = flist[base + u];
                        unsigned long long ff = fprev[m];
                        const unsigned long long sv = sprev[m];
                        if (j < rows) {
                            while (ff) {
                                const int r = __ffsll((long long)ff) - 1;
                                ff &= ff - 1;
                                Hs[r * a.rows_per + j] += (((sv >> r) & 1ull) ? 2 : -2) * jv[u];
                            }
                        }
                    }
                }
                __syncthreads();
                }
            }
            // ---- publish block q+1 (TCU: the tiles while the MMAs run, the fields after them)
            if constexpr (TCU) {
                if (q + 1 < total) tile_flush(q + 1);
                __syncthreads();   // every thread is past its reads of ring slot q-1 (= slot q+3)
                if (pn3_ok) ring_slot(q + 3)[threadIdx.x] = pn3;
                if (q + 1 < total) {
                    // owned positions of block q+1
                    const int32_t *Pn = ring_slot(q + 1);
                    const int32_t cnt = block_cnt(q + 1);
                    if (threadIdx.x == 0) s_nown = 0;
                    __syncthreads();
                    if ((int)threadIdx.x < cnt) {
                        const int32_t p = Pn[threadIdx.x];
                        if (p >= ua && p < ub) ownl[atomicAdd(&s_nown, 1)] = (int32_t)threadIdx.x;
                    }
                    __syncthreads();
                    Pnext = ring_slot(q + 1);
                }
                if (issued) {
                    if (!mbar_wait(&s_mbar, mphase & 1u)) {
                        atomicCAS(&a.ctl->err, 0, (int)PAMC_ERR_TIMEOUT);
                        mbar_wait(&s_mbar, mphase & 1u);
                    }
                    ++mphase;
                    tc_fence_after();
                }
                if (q + 1 < total) publish_G(q + 1);
            } else if (q + 1 < total) {
                publish_lists(q + 1);
                publish_G(q + 1);
                publish_tiles(q + 1);
            }
        } else if (q < total) {
            const int32_t cnt = block_cnt(q);
            const int32_t cntp = q > 0 ? block_cnt(q - 1) : 0;
            const int32_t nstg = min(s_nslot, kStgSlots);          // rows staged by the last chain
            // block q+1's mode (written in phase q-1), consumed after the prep
            const int32_t t2_next = __ldcg(&a.bar->t2_mode[(q + 1) & 3]);
            if ((int)threadIdx.x < cnt) Pc[threadIdx.x] = pcn;   // loaded last phase
            // positions of block q+1, for staging rows during this chain
            const int32_t q1 = min(q + 1, total - 1);
            const int32_t pnx_v = block_pos(q1)[min((int32_t)threadIdx.x, block_cnt(q1) - 1)];
            if (blockIdx.x == a.n_upd && threadIdx.x < kB) {   // buffer of block q+1 starts empty
                a.flip[((q + 1) % 3) * kB + threadIdx.x] = 0ull;
                a.snew[((q + 1) % 3) * kB + threadIdx.x] = 0ull;
            }
            // the independent loads first: the published fields, block q-1's
            // flip masks and the two tiles; they complete while the
            // thresholds are computed
            // (unconditional loads from clamped indices: nothing waits for
            // them until they are stored after the thresholds).  A position's
            // four fields of the group are 16 contiguous bytes.
            const int32_t *Gq = a.G + (size_t)(q & 1) * kB * 64;
            const int4 g4 = *reinterpret_cast<const int4 *>(Gq + (size_t)min((int32_t)threadIdx.x, cnt - 1) * 64 + cg * 4);
            const bool okm = q > 0 && (int)threadIdx.x < cntp;
            const size_t mi = (size_t)(q > 0 ? (q - 1) % 3 : 0) * kB + min((int32_t)threadIdx.x, kB - 1);
            const unsigned long long fm = a.flip[mi], sm2 = a.snew[mi];
            {
                const uint32_t *Tq = a.T + (size_t)(q & 1) * kB * kC;
                const uint32_t *T2q = a.T2 + (size_t)(q & 1) * kB * kC;
                const bool t2_global = q > 0 && t2_cur;
                for (int32_t x = threadIdx.x; x < kB * kC / 4; x += blockDim.x) {
                    cp_async16(tile + (size_t)x * 4, Tq + (size_t)x * 4);
                    if (t2_global) cp_async16(tile2 + (size_t)x * 4, T2q + (size_t)x * 4);
                }
                cp_async_commit();
            }
            // rows loaded at the end of the last chain (no-op otherwise): after
            // the loads above are on their way, so the waits overlap
            chain_t2_flush();
            if ((int)threadIdx.x < kB) gmask[threadIdx.x] = 0u;
            cp_async_wait_prior();   // this thread's staged pieces (all but the tiles just issued)
            __syncthreads();   // Pc, staged pieces
            if (threadIdx.x == 0) s_nslot = 0;
            // staged rows of the last block's flips -> bit rows of J[P_{q-1}][P_q]
            for (int32_t task = warp; task < nstg * kC; task += kSwThreads / 32) {   // warp-uniform
                const int32_t sl = task / kC, wv = task % kC, m2 = wv * 32 + lane;
                const uint32_t piece = stg[(size_t)task * 32 + lane];
                const int32_t col = Pc[min(m2, cnt - 1)];
                const uint32_t raw = (piece >> (8 * (col & 3))) & 0xFFu;
                const uint32_t word = __ballot_sync(0xffffffffu, m2 < cnt && e4m3_pm1(raw) > 0);
                if (lane == 0) tile2[(size_t)Uslot[sl] * kC + wv] = word;
            }
            if (q == 0) thresholds(0, Pc, 0, blockDim.x, 0);   // later blocks: computed during the last chain
            if ((int)threadIdx.x < cnt) {
                const int32_t m = threadIdx.x;
                Gs[m] = cg * 4 < R ? g4.x : 0;
                Gs[kB + m] = cg * 4 + 1 < R ? g4.y : 0;
                Gs[2 * kB + m] = cg * 4 + 2 < R ? g4.z : 0;
                Gs[3 * kB + m] = cg * 4 + 3 < R ? g4.w : 0;
            }
            if (okm) { cfm[threadIdx.x] = fm; csn[threadIdx.x] = sm2; }
            if ((int)threadIdx.x < kB) Pnx[threadIdx.x] = pnx_v;
            cp_async_wait_all();
            __syncthreads();
            // positions of block q+1 for the next phase (unconditional, from a
            // clamped index: nothing waits for them here)
            if (q + 1 < total) pcn = block_pos(q + 1)[min((int32_t)threadIdx.x, block_cnt(q + 1) - 1)];
            if (warp < 4 && cg * 4 + warp < R) {
                const bool pf_rows = q + 1 < total && !t2_next && stage_ok;
                const int32_t cnt1 = block_cnt(q1);
                const int qq = warp;
                const int r = cg * 4 + qq;
                uint32_t *bits = cbits + (size_t)qq * nw;
                int32_t f[kC], th[kC];
                uint32_t smask[kC];
#pragma unroll
                for (int s2 = 0; s2 < kC; ++s2) {
                    const int32_t m = s2 * 32 + lane;
                    const bool ok = m < cnt;
                    f[s2] = ok ? Gs[qq * kB + m] : 0;
                    th[s2] = ok ? thr_all[(size_t)(q & 1) * 4 * kB + qq * kB + m] : 0;
                    const int32_t k = ok ? Pc[m] : 0;
                    smask[s2] = __ballot_sync(0xffffffffu, ok && ((bits[k >> 5] >> (k & 31)) & 1u));
                }
                // block q-1's flips, which the published fields do not include yet.
                // Blocks of one sweep are disjoint; at a seam (block q-1 ends the
                // previous sweep) the two blocks can share vertices
                if (q > 0) {
                    const bool seam = (q % nb) == 0;
                    const int32_t *Pprv = block_pos(q - 1);
#pragma unroll
                    for (int s2 = 0; s2 < kC; ++s2) {
                        const int32_t mp = s2 * 32 + lane;
                        unsigned int bal =
                            __ballot_sync(0xffffffffu, mp < cntp && ((cfm[mp] >> r) & 1ull));
                        while (bal) {
                            const int o = __ffs(bal) - 1;
                            bal &= bal - 1;
                            const int32_t m = s2 * 32 + o;
                            const int32_t d = ((csn[m] >> r) & 1ull) ? 2 : -2;
                            const uint4 t0 = *reinterpret_cast<const uint4 *>(tile2 + (size_t)m * kC);
                            const uint4 t1 = *reinterpret_cast<const uint4 *>(tile2 + (size_t)m * kC + 4);
                            const uint32_t tw[kC] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
                            for (int s3 = 0; s3 < kC; ++s3) f[s3] += ((tw[s3] >> lane) & 1u) ? d : -d;
                            if (seam) {
                                // J_vv = 0 where the vertex is also in block q: undo the -d of its clear bit
                                const int32_t v = Pprv[m];
#pragma unroll
                                for (int s3 = 0; s3 < kC; ++s3)
                                    if (s3 * 32 + lane < cnt && Pc[s3 * 32 + lane] == v) f[s3] += d;
                            }
                        }
                    }
                }
                // the sequential decisions of block q, 32 positions at a time:
                // every lane evaluates its own position with the current
                // fields; positions before the first lane that flips keep their
                // spins, that flip is applied to all fields, and evaluation
                // resumes after it -- the same result as one position at a time
#pragma unroll
                for (int s2 = 0; s2 < kC; ++s2) {
                    const int32_t mb = s2 * 32;
                    if (mb >= cnt) break;
                    const uint32_t sold = (smask[s2] >> lane) & 1u;
                    unsigned int open = cnt - mb >= 32 ? 0xffffffffu : ((1u << (cnt - mb)) - 1u);
                    while (open) {
                        uint32_t snv;
                        if (a.rule == 0) {
                            snv = f[s2] >= th[s2] ? 1u : 0u;
                        } else {
                            const int32_t x = sold ? f[s2] : -f[s2];
                            snv = x <= th[s2] ? (sold ^ 1u) : sold;
                        }
                        const unsigned int fb = __ballot_sync(0xffffffffu, snv != sold) & open;
                        if (fb == 0u) break;
                        const int o = __ffs(fb) - 1;
                        open &= ~((2u << o) - 1u);        // positions up to o are decided
                        const int32_t m = mb + o;
                        const int32_t d = ((smask[s2] >> o) & 1u) ? -2 : 2;   // the spin turns over
                        // (the diagonal bit is arbitrary: position m is decided)
                        const uint4 t0 = *reinterpret_cast<const uint4 *>(tile + (size_t)m * kC);
                        const uint4 t1 = *reinterpret_cast<const uint4 *>(tile + (size_t)m * kC + 4);
                        const uint32_t tw[kC] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
                        for (int s3 = 0; s3 < kC; ++s3) f[s3] += ((tw[s3] >> lane) & 1u) ? d : -d;
                        uint32_t before = 1u;
                        int32_t slot = kStgSlots;
                        if (lane == 0) {
                            const int32_t k = Pc[m];
                            bits[k >> 5] ^= 1u << (k & 31);
                            before = atomicOr(&gmask[m], 1u << qq);
                            atomicOr(&a.flip[(q % 3) * kB + m], 1ull << r);
                            if (d > 0) atomicOr(&a.snew[(q % 3) * kB + m], 1ull << r);
                            if (pf_rows && before == 0u) {
                                slot = atomicAdd(&s_nslot, 1);
                                if (slot < kStgSlots) Uslot[slot] = m;
                            }
                        }
                        // few flips: the first replica of the group to flip at m pulls
                        // m's coupling row into L2 for the next phase's field update and
                        // stages the pieces of it over the next block's positions
                        if (pf_rows && __shfl_sync(0xffffffffu, before, 0) == 0u) {
                            const uint8_t *row = a.J + (size_t)Pc[m] * n;
                            for (int32_t off = lane * 128; off < n; off += 32 * 128)
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(row + off));
                            slot = __shfl_sync(0xffffffffu, slot, 0);
                            if (slot < kStgSlots) {
#pragma unroll
                                for (int wv = 0; wv < kC; ++wv) {
                                    const int32_t m2 = wv * 32 + lane;
                                    if (m2 < cnt1)
                                        cp_async4(stg + ((size_t)slot * kC + wv) * 32 + lane, row + (Pnx[m2] & ~3));
                                }
                            }
                        }
                    }
                }
            } else if (warp >= 4 && warp < 12 && q + 1 < total) {
                // eight of the idle warps: the next block's thresholds (they
                // depend on the draws only)
                thresholds(q + 1, block_pos(q + 1), 128, 256, 2);
            }
            t2_cur = t2_next;   // block q+1 is the next block
        }
        // the update CTAs produce block q+2's J[P_{q+1}][P_{q+2}] unless block
        // q-1 had few flipped positions (always with the CUDA-core update)
        const bool t2_on = !TCU || q == 0 || nl_q > kT2Rare;
        if (upd && blockIdx.x == 0 && threadIdx.x == 0 && q + 2 < total) a.bar->t2_mode[(q + 2) & 3] = t2_on;
        // chain CTAs: block q decided; if block q+1's tile is not produced, its
        // rows were staged during the chain -- unless more positions flipped
        // than there are slots: then the rows of all of them are loaded here
        if (!upd && q < total) cp_async_commit();   // the staged pieces
        bool t2_load = false;
        if (!upd && q + 1 < total && !t2_cur) {
            __syncthreads();   // the decisions (gmask, the staging count) are complete
            t2_load = !stage_ok || s_nslot > kStgSlots;
        }
        if (t2_load) {
            const int32_t cnt1 = block_cnt(q + 1);
            if ((int)threadIdx.x < cnt1) Pnx[threadIdx.x] = pcn;
            if (threadIdx.x == 0) s_nu = 0;
            __syncthreads();
            if ((int)threadIdx.x < block_cnt(q) && gmask[threadIdx.x] != 0u) Ulist[atomicAdd(&s_nu, 1)] = threadIdx.x;
            __syncthreads();
            chain_t2_issue(s_nu, cnt1);
        }
        grid_arrive(a.bar);
        if (upd && TCU) tile_issue(q + 2, t2_on ? kTileWords : kTileWordsT);
        if (!grid_wait(a.bar, nblocks, gen, a.ctl, &s_ok)) { alive = false; break; }
    }

    // ---------------- energies E_r = -1/2 sum_j s_j h_j, fields and spins back to HBM
    if (upd && TCU) {
        if (alive) {
            const int quarter = warp & 3;
            for (int32_t pr = warp >> 2; pr < a.ntiles * 4; pr += (kSwThreads / 32) / 4) {
                const int tile = pr >> 2, c0 = (pr & 3) * 16;
                const int32_t ar = tile * 128 + quarter * 32 + lane;
                const int32_t j = tu_row_of(ar);
                uint32_t v[16];
                tc_ld16(s_tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tile * 64 + c0), v);
                const int32_t s01 = j < rows ? 1 : 0;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int r = c0 + c;
                    const int32_t hv = __float2int_rn(__uint_as_float(v[c]));
                    long long accv = 0;
                    if (s01 && r < R) {
                        a.H[(size_t)r * n + ua + j] = hv;
                        const int32_t sgn = ((ubits[r * rw + (j >> 5)] >> (j & 31)) & 1u) ? 1 : -1;
                        accv = (long long)sgn * hv;
                    }
                    for (int o = 16; o > 0; o >>= 1) accv += __shfl_down_sync(0xffffffffu, accv, o);
                    if (lane == 0 && r < R && accv != 0) atomicAdd((unsigned long long *)&a.E[r], (unsigned long long)accv);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        if (warp == 0) tc_dealloc(s_tmem, kTuCols);
    } else if (!alive) {
        return;
    } else if (upd) {
        for (int32_t x = threadIdx.x; x < R * rows; x += blockDim.x) {
            const int r = x / rows, j = x % rows;
            a.H[(size_t)r * n + ua + j] = Hs[r * a.rows_per + j];
        }
        for (int r = 0; r < R; ++r) {
            long long accv = 0;
            for (int32_t j = threadIdx.x; j < rows; j += blockDim.x) {
                const int32_t s = ((ubits[r * rw + (j >> 5)] >> (j & 31)) & 1u) ? 1 : -1;
                accv += (long long)s * Hs[r * a.rows_per + j];
            }
            for (int o = 16; o > 0; o >>= 1) accv += __shfl_down_sync(0xffffffffu, accv, o);
            if (lane == 0 && accv != 0) atomicAdd((unsigned long long *)&a.E[r], (unsigned long long)accv);
        }
    } else {
        for (int32_t x = threadIdx.x; x < 4 * n; x += blockDim.x) {
            const int qq = x / n;
            const int32_t k = x % n;
            const int r = cg * 4 + qq;
            if (r < R) a.dst[(size_t)r * n + k] = ((cbits[qq * nw + (k >> 5)] >> (k & 31)) & 1u) ? 1 : -1;
        }
    }
}

// E_r = -1/2 sum_j s_j h_j from recomputed fields (one CTA per replica)
__global__ void k_dense_energy_from_H(int32_t n, const int32_t *__restrict__ H,
                                      const int8_t *__restrict__ spins, int64_t *__restrict__ E,
                                      const DevCtl *__restrict__ ctl, int restart_t) {
    __shared__ long long red[32];
    if (restart_t >= 0 ? !(ctl->restart && ctl->t == restart_t) : ctl->done != 0) return;
    const int r = blockIdx.x;
    long long acc = 0;
    for (int32_t j = threadIdx.x; j < n; j += blockDim.x)
        acc += (long long)spins[(size_t)r * n + j] * H[(size_t)r * n + j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        E[r] = -(tot / 2);
    }
}

// Max-Cut weights -> couplings in place (J = -w), and W = sum_{i<j} w_ij.
__global__ void k_dense_negate_sum(size_t total, int8_t *__restrict__ J,
                                   unsigned long long *__restrict__ wsum) {
    long long acc = 0;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
         x += (size_t)gridDim.x * blockDim.x) {
        const int8_t v = J[x];
        acc += v;
        J[x] = (int8_t)(-v);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0) atomicAdd(wsum, (unsigned long long)acc);
}

// the accumulated sum_j s_j h_j becomes E = -sum/2
__global__ void k_dense_energy_finish(int32_t R, int64_t *E, const DevCtl *ctl) {
    if (ctl->done) return;
    const int r = threadIdx.x;
    if (r < R) E[r] = -(E[r] / 2);
}

// int8 couplings (validated +-1 / 0) -> e4m3 bytes in place
__global__ void k_dense_to_e4m3(size_t total, uint8_t *__restrict__ J) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
         x += (size_t)gridDim.x * blockDim.x) {
        const int8_t v = (int8_t)J[x];
        J[x] = v == 0 ? (uint8_t)0 : (v > 0 ? (uint8_t)0x38 : (uint8_t)0xB8);
    }
}

// Validation of a device-resident copy: entries in {-1, 0, +1}, zero diagonal,
// +-1 off the diagonal, symmetric.  32x32 tiles compared with their transpose.
__global__ void k_dense_validate(int32_t n, const int8_t *__restrict__ J, int *__restrict__ err) {
    __shared__ int8_t tl[32][33];
    const int32_t bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    if (bj < bi) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int yy = ty; yy < 32; yy += blockDim.x / 32) {
        const int32_t i = bj + yy, j = bi + tx;
        tl[yy][tx] = (i < n && j < n) ? J[(size_t)i * n + j] : 0;
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += blockDim.x / 32) {
        const int32_t i = bi + yy, j = bj + tx;
        if (i < n && j < n) {
            const int8_t v = J[(size_t)i * n + j];
            if (i == j) { if (v != 0) atomicCAS(err, 0, (int)PAMC_ERR_DIAG); }
            else if (v != 1 && v != -1) atomicCAS(err, 0, (int)PAMC_ERR_RANGE);
            else if (v != tl[tx][yy]) atomicCAS(err, 0, (int)PAMC_ERR_ASYM);
        }
    }
}

}  // namespace

cudaError_t launch_dense_validate(int32_t n, const int8_t *J, int *err, cudaStream_t st) {
    const int nt = (n + 31) / 32;
    k_dense_validate<<<dim3(nt, nt), 256, 0, st>>>(n, J, err);
    return cudaGetLastError();
}

cudaError_t launch_dense_perm(int32_t n, uint64_t seed, int32_t t, int32_t S, int32_t *perm,
                              uint32_t *skey, int32_t *sidx, int32_t *boff, const DevCtl *ctl, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    k_dense_perm_bucket<<<S, kPermThreads, 0, st>>>(n, (uint32_t)seed, (uint32_t)(seed >> 32), t, skey, sidx,
                                                   boff, ctl);
    k_dense_perm_sort<<<dim3((1 << kPermBucketBits) / kSortBuckets, S), 256, 0, st>>>(n, skey, sidx, boff, perm,
                                                                                       ctl);
    return cudaGetLastError();
}

size_t dense_perm_offsets(int32_t S) { return (size_t)S * ((1 << kPermBucketBits) + 1); }

cudaError_t launch_dense_tables(int rule, int32_t Hc, int32_t n, DevCtl *ctl, uint64_t *tab,
                                cudaStream_t st) {
    const int32_t cntv = rule == 0 ? 2 * Hc + 1 : Hc + 1;
    int grid = (cntv + 255) / 256;
    if (grid > 304) grid = 304;
    k_dense_tables<<<grid, 256, 0, st>>>(rule, Hc, n, ctl, tab);
    return cudaGetLastError();
}

size_t dense_recompute_smem() { return (size_t)kRcStages * kRcStageBytes; }

cudaError_t launch_dense_recompute(int32_t n, int32_t R, const int8_t *J, const int8_t *src,
                                   const int32_t *parent, const int8_t *ncm_buf,
                                   const int32_t *ncm_idx, int32_t *H, const DevCtl *ctl,
                                   cudaStream_t st, int restart_t) {
    const size_t smem = dense_recompute_smem();
    cudaError_t e = allow_dynamic_smem(k_dense_recompute, smem);
    if (e != cudaSuccess) return e;
    const int grid = (n + kRcRows - 1) / kRcRows;
    k_dense_recompute<<<grid, kRcWarps * 32, smem, st>>>(n, R, reinterpret_cast<const uint8_t *>(J), src,
                                                           parent, ncm_buf, ncm_idx, H, ctl, restart_t);
    return cudaGetLastError();
}

cudaError_t launch_dense_energy(int32_t n, int32_t R, const int32_t *H, const int8_t *spins, int64_t *E,
                                const DevCtl *ctl, cudaStream_t st, int restart_t) {
    k_dense_energy_from_H<<<R, 512, 0, st>>>(n, H, spins, E, ctl, restart_t);
    return cudaGetLastError();
}

cudaError_t launch_dense_to_e4m3(size_t total, int8_t *J, cudaStream_t st) {
    k_dense_to_e4m3<<<152 * 8, 256, 0, st>>>(total, reinterpret_cast<uint8_t *>(J));
    return cudaGetLastError();
}

cudaError_t launch_dense_negate_sum(size_t total, int8_t *J, unsigned long long *wsum, cudaStream_t st) {
    k_dense_negate_sum<<<152 * 8, 256, 0, st>>>(total, J, wsum);
    return cudaGetLastError();
}

int dense_block_positions() { return kB; }

// Shared memory of the sweep kernel for a given split.
size_t dense_sweep_smem(int32_t n, int32_t R, int32_t rows_per, bool tcu) {
    const size_t rest = ((((size_t)R * ((rows_per + 31) / 32) * 4) + 15) & ~(size_t)15) +
                        (size_t)kB * (8 + 8 + 4 + 16 + 4 + 4);
    const size_t ntiles = ((size_t)rows_per + 127) / 128;
    const size_t upd = tcu ? 1024 + 2 * ntiles * kTuTileBytes + 2 * kTuBSlice + rest
                           : (((size_t)R * rows_per * 4 + 15) & ~(size_t)15) + rest;
    const size_t nw = (size_t)((n + 31) / 32);
    const size_t chn = 2 * (size_t)kB * kC * 4 + ((4 * nw + 3) & ~(size_t)3) * 4 + (size_t)kWin * 8 +
                       (size_t)kB * (4 * 4 + 8 * 4 + 4 + 8 + 8 + 16 + 12) +
                       (size_t)kStgSlots * (kC * 32 * 4 + 4);
    return upd > chn ? upd : chn;
}

cudaError_t launch_dense_sweep(int32_t n, int32_t R, int32_t S, int32_t rule, int32_t Hc, int32_t t,
                               uint64_t seed, int32_t n_upd, int32_t rows_per, int32_t grid,
                               const int8_t *J, const int32_t *perm, const uint64_t *tab,
                               const int8_t *src, const int32_t *parent, const int8_t *ncm_buf,
                               const int32_t *ncm_idx, int32_t *H, int8_t *dst, int64_t *E,
                               int32_t *G, uint32_t *T, uint32_t *T2, unsigned long long *flip,
                               unsigned long long *snew, void *bar, DevCtl *ctl, cudaStream_t st, bool tcu,
                               int32_t rbase) {
    DenseSweepArgs a;
    a.n = n; a.R = R; a.S = S; a.rule = rule; a.Hc = Hc; a.n_upd = n_upd; a.rows_per = rows_per;
    a.ntiles = (rows_per + 127) / 128;
    a.t = t; a.K = make_philox_keys(seed); a.J = reinterpret_cast<const uint8_t *>(J); a.perm = perm;
    a.tab = tab; a.src = src; a.parent = parent; a.ncm_buf = ncm_buf; a.ncm_idx = ncm_idx; a.H = H;
    a.dst = dst; a.E = E; a.G = G; a.T = T; a.T2 = T2; a.flip = flip; a.snew = snew;
    a.bar = reinterpret_cast<GridBar *>(bar); a.ctl = ctl;
    a.gbase = rbase / 4;
    if (tcu && (a.ntiles > kTuMaxTiles || n % 16 != 0 || rows_per % 32 != 0)) return cudaErrorInvalidValue;
    const size_t smem = dense_sweep_smem(n, R, rows_per, tcu);
    const void *fn = tcu ? (const void *)k_dense_sweep<true> : (const void *)k_dense_sweep<false>;
    cudaError_t e = tcu ? allow_dynamic_smem(k_dense_sweep<true>, smem) : allow_dynamic_smem(k_dense_sweep<false>, smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(bar, 0, sizeof(GridBar), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kSwThreads), args, smem, st);
    if (e != cudaSuccess) return e;
    k_dense_energy_finish<<<1, 64, 0, st>>>(R, E, ctl);
    return cudaGetLastError();
}

int dense_sweep_threads() { return kSwThreads; }

}  // namespace pamc
