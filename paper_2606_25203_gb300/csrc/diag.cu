// diag.cu -- population diversity: the pairwise Hamming distance between
// replica configurations, corrected for the global spin-flip symmetry of
// Max-Cut, d_H = min(d, n - d) (Suppl., Hamming distance of replicas).
//
// On the tensor cores (the default): the overlaps G = S S^T of the +-1
// population are an exact fp8 contraction (+-1 is exact in e4m3, partial sums
// are integers below 2^24 in the fp32 accumulator), and d = (n - G_rr') / 2.
// A CTA owns 256 rows i (two M=128 tiles) and 64 columns j of G; TMA copies
// 128-byte K slices of both row sets (128-byte swizzle, three stages), one
// thread issues tcgen05.mma kind::f8f6f4 into tensor memory, and four warps
// read the accumulator back and count the pairs i < j of their block into a
// shared-memory histogram, flushed once per CTA.
//
// On the CUDA cores (PAMC_HAMMING=cuda, or where tensor maps are
// unavailable): the +-1 spins are packed one bit per spin (a warp ballot per
// 32 spins of a row), then every pair r < r' is counted by XOR and popcount
// over the packed words, tile by tile: a CTA owns a 32 x 32 block of pairs
// and stages 32 words of both row sets in shared memory per round.  Results
// are exact integers: a histogram over the corrected distance and its sum.
#include <cuda.h>

#include <cstdlib>
#include <cstring>

#include "pamc_device.cuh"
#include "pamc_internal.h"
#include "tc_sm100.cuh"

namespace pamc {

namespace {

constexpr int kTile = 32;    // replicas per tile side
constexpr int kWords = 32;   // packed words staged per round

// bits[r][w] bit b = (spins[r][32w + b] > 0); one warp per (r, w)
__global__ void k_pack_bits(const int8_t *__restrict__ spins, int32_t R, int32_t n, int32_t nw,
                            uint32_t *__restrict__ bits) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= (int64_t)R * nw) return;
    const int32_t r = (int32_t)(warp / nw), w = (int32_t)(warp % nw);
    const int32_t k = w * 32 + lane;
    const bool up = k < n && spins[(size_t)r * n + k] > 0;
    const uint32_t word = __ballot_sync(0xffffffffu, up);
    if (lane == 0) bits[(size_t)r * nw + w] = word;
}

// One CTA per tile (bi <= bj) of 32 x 32 replica pairs; 256 threads, each
// thread four pairs (one row i, four columns j).
__global__ void __launch_bounds__(256)
k_hamming(const uint32_t *__restrict__ bits, int32_t R, int32_t n, int32_t nw, int32_t ntiles,
          unsigned long long *__restrict__ hist, unsigned long long *__restrict__ sum) {
    __shared__ uint32_t A[kTile][kWords + 1];
    __shared__ uint32_t B[kTile][kWords + 1];
    __shared__ unsigned long long red[8];
    // tile index -> (bi, bj), bi <= bj, row-major over the upper triangle
    int32_t q = blockIdx.x, bi = 0;
    while (q >= ntiles - bi) { q -= ntiles - bi; ++bi; }
    const int32_t bj = bi + q;
    const int32_t i0 = bi * kTile, j0 = bj * kTile;
    const int ti = threadIdx.x >> 3;          // row of the tile, 0..31
    const int tj = (threadIdx.x & 7) * 4;     // first of four columns
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
    for (int32_t w0 = 0; w0 < nw; w0 += kWords) {
        for (int x = threadIdx.x; x < kTile * kWords; x += blockDim.x) {
            const int rr = x / kWords, ww = x % kWords;
            const int32_t w = w0 + ww;
            A[rr][ww] = (i0 + rr < R && w < nw) ? bits[(size_t)(i0 + rr) * nw + w] : 0u;
            B[rr][ww] = (j0 + rr < R && w < nw) ? bits[(size_t)(j0 + rr) * nw + w] : 0u;
        }
        __syncthreads();
#pragma unroll 8
        for (int ww = 0; ww < kWords; ++ww) {
            const uint32_t a = A[ti][ww];
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] += __popc(a ^ B[tj + c][ww]);
        }
        __syncthreads();
    }
    unsigned long long local = 0;
    const int32_t i = i0 + ti;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int32_t j = j0 + tj + c;
        if (i < R && j < R && i < j) {
            const int32_t d = (int32_t)acc[c];
            const int32_t dc = d < n - d ? d : n - d;
            atomicAdd(&hist[dc], 1ull);
            local += (unsigned long long)dc;
        }
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int x = 0; x < 8; ++x) s += red[x];
        atomicAdd(sum, s);
    }
}

// ---------------------------------------------------------------- tensor cores
constexpr int kHtRows = 256;                  // rows i per CTA (two M=128 tiles)
constexpr int kHtCols = 64;                   // columns j per CTA (N)
constexpr int kHtKB = 128;                    // K bytes per slice (one swizzle atom)
constexpr int kHtStages = 3;
constexpr int kHtABytes = kHtRows * kHtKB;
constexpr int kHtBBytes = kHtCols * kHtKB;
constexpr int kHtStageBytes = kHtABytes + kHtBBytes;
constexpr int kHtThreads = 128;
constexpr uint32_t kHtTmemCols = 128;         // two tiles x N=64 fp32 columns
constexpr int32_t kHtHistBins = 16384;        // histogram bins kept in shared memory (n <= 32,766)
// instruction descriptor: D f32, A and B e4m3, both K-major, N=64, M=128
constexpr uint32_t kHtIdesc = (1u << 4) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// Sb[r][k] = +-1.0 in e4m3 for r < R, k < n; 0 in the padding
__global__ void k_pm1_e4m3(int32_t n, int32_t n_pad, int32_t R, int32_t R_pad, const int8_t *__restrict__ spins,
                           uint8_t *__restrict__ Sb) {
    const size_t total = (size_t)R_pad * n_pad;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)(x / n_pad), k = (int32_t)(x % n_pad);
        uint8_t v = 0;
        if (r < R && k < n) v = spins[(size_t)r * n + k] > 0 ? 0x38u : 0xB8u;
        Sb[x] = v;
    }
}

__global__ void __launch_bounds__(kHtThreads, 1)
k_hamming_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int32_t n,
             int32_t n_pad, int32_t R, unsigned long long *__restrict__ hist, unsigned long long *__restrict__ sum,
             int *__restrict__ err) {
    const int32_t i0 = blockIdx.x * kHtRows, j0 = blockIdx.y * kHtCols;
    if (j0 + kHtCols - 1 <= i0) return;   // every pair of the block has i >= j
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[kHtStages], empty[kHtStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;
    __shared__ unsigned long long red[kHtThreads / 32];
    uint8_t *base = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
    uint32_t *hs = reinterpret_cast<uint32_t *>(base + (size_t)kHtStages * kHtStageBytes);
    const int32_t nbins = n / 2 + 1;
    const bool hsm = nbins <= kHtHistBins;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t nk = (n_pad + kHtKB - 1) / kHtKB;
    if (hsm)
        for (int32_t b = threadIdx.x; b < nbins; b += blockDim.x) hs[b] = 0u;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kHtStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(&done, 1);
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc_alloc(&tmem_base, kHtTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer: slice kc into stage kc % kHtStages once its previous MMAs completed
        int32_t issued = 0;
        for (int32_t kc = 0; kc < nk; ++kc) {
            const int s = kc % kHtStages;
            const int32_t round = kc / kHtStages;
            if (round > 0 && !mbar_wait(&empty[s], (uint32_t)((round - 1) & 1))) {
                atomicCAS(err, 0, (int)PAMC_ERR_TIMEOUT);
                s_err = 1;
                break;
            }
            if (*(volatile int *)&s_err) break;
            uint8_t *A = base + (size_t)s * kHtStageBytes;
            mbar_expect_tx(&full[s], (uint32_t)kHtStageBytes);
            tma_load_2d(A, &tmA, kc * kHtKB, i0, &full[s]);
            tma_load_2d(A + kHtABytes, &tmB, kc * kHtKB, j0, &full[s]);
            issued = kc + 1;
        }
        for (int32_t kc = (issued > kHtStages ? issued - kHtStages : 0); kc < issued; ++kc)
            mbar_wait(&full[kc % kHtStages], (uint32_t)((kc / kHtStages) & 1));
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int32_t kc = 0; kc < nk; ++kc) {
            const int s = kc % kHtStages;
            if (!mbar_wait(&full[s], (uint32_t)((kc / kHtStages) & 1)) || *(volatile int *)&s_err) {
                atomicCAS(err, 0, (int)PAMC_ERR_TIMEOUT);
                s_err = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(base + (size_t)s * kHtStageBytes);
            const uint32_t b0 = a0 + kHtABytes;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int ks = 0; ks < kHtKB / 32; ++ks)
                    tc_mma(tmem + (uint32_t)(mt * 64), sw128_desc(a0 + mt * 128 * kHtKB) + (uint64_t)(2 * ks),
                           sw128_desc(b0) + (uint64_t)(2 * ks), kHtIdesc, (kc > 0 || ks > 0) ? 1u : 0u);
            tc_commit(&empty[s]);
        }
        tc_commit(&done);
    }
    __syncwarp();
    // epilogue: warp w holds rows 32w .. 32w+31 of each M tile in its lanes
    const bool ok = mbar_wait(&done, 0u);
    tc_fence_after();
    unsigned long long local = 0;
    if (ok && !*(volatile int *)&s_err) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int32_t i = i0 + mt * 128 + warp * 32 + lane;
#pragma unroll
            for (int c0 = 0; c0 < kHtCols; c0 += 16) {
                uint32_t v[16];
                tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * 64 + c0), v);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int32_t j = j0 + c0 + jj;
                    if (i < j && j < R) {
                        const int32_t g = __float2int_rn(__uint_as_float(v[jj]));   // overlap, n - 2 d
                        const int32_t d = (n - g) >> 1;
                        const int32_t dc = d < n - d ? d : n - d;
                        if (hsm) atomicAdd(&hs[dc], 1u);
                        else atomicAdd(&hist[dc], 1ull);
                        local += (unsigned long long)dc;
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicCAS(err, 0, (int)PAMC_ERR_TIMEOUT);
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if (lane == 0) red[warp] = local;
    tc_fence_before();
    __syncthreads();
    if (hsm)
        for (int32_t b = threadIdx.x; b < nbins; b += blockDim.x)
            if (hs[b] != 0u) atomicAdd(&hist[b], (unsigned long long)hs[b]);
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < kHtThreads / 32; ++w) tot += red[w];
        if (tot) atomicAdd(sum, tot);
    }
    if (warp == 0) tc_dealloc(tmem, kHtTmemCols);
}

}  // namespace

size_t hamming_tc_scratch(int32_t n, int32_t R) {
    const size_t n_pad = ((size_t)n + 15) & ~(size_t)15;
    const size_t R_pad = ((size_t)R + kHtRows - 1) / kHtRows * kHtRows;
    return n_pad * R_pad;
}

bool hamming_tc_enabled(int32_t n, int32_t R) {
    const char *env = getenv("PAMC_HAMMING");
    if (env && strcmp(env, "cuda") == 0) return false;
    return R >= 2 && n >= 1 && dense_tc_supported(16);
}

cudaError_t launch_hamming_tc(int32_t n, int32_t R, const int8_t *spins, uint8_t *Sb, unsigned long long *hist,
                              unsigned long long *sum, int *err, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * ((size_t)n / 2 + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sum, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || R < 2) return e;
    const int32_t n_pad = (n + 15) & ~15;
    const int32_t R_pad = (R + kHtRows - 1) / kHtRows * kHtRows;
    alignas(64) unsigned char mapA[128], mapB[128];
    e = dense_tc_map(mapA, Sb, R_pad, n_pad, kHtRows);
    if (e == cudaSuccess) e = dense_tc_map(mapB, Sb, R_pad, n_pad, kHtCols);
    if (e != cudaSuccess) return e;
    const size_t total = (size_t)R_pad * n_pad;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    k_pm1_e4m3<<<grid, 256, 0, st>>>(n, n_pad, R, R_pad, spins, Sb);
    const size_t smem = (size_t)kHtStages * kHtStageBytes + 1024 +
                        ((n / 2 + 1) <= kHtHistBins ? (size_t)(n / 2 + 1) * 4 : 0);
    e = allow_dynamic_smem(k_hamming_tc, smem);
    if (e != cudaSuccess) return e;
    const dim3 g2(R_pad / kHtRows, (R + kHtCols - 1) / kHtCols);
    k_hamming_tc<<<g2, kHtThreads, smem, st>>>(*reinterpret_cast<const CUtensorMap *>(mapA),
                                                *reinterpret_cast<const CUtensorMap *>(mapB), n, n_pad, R, hist, sum,
                                                err);
    return cudaGetLastError();
}

cudaError_t launch_hamming(int32_t n, int32_t R, const int8_t *spins, uint32_t *bits,
                           unsigned long long *hist, unsigned long long *sum, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * ((size_t)n / 2 + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sum, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || R < 2) return e;
    const int32_t nw = (n + 31) / 32;
    const int64_t warps = (int64_t)R * nw;
    k_pack_bits<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(spins, R, n, nw, bits);
    const int32_t nt = (R + kTile - 1) / kTile;
    const int64_t tiles = (int64_t)nt * (nt + 1) / 2;
    k_hamming<<<(unsigned)tiles, 256, 0, st>>>(bits, R, n, nw, nt, hist, sum);
    return cudaGetLastError();
}

}  // namespace pamc
