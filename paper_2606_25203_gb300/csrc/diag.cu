// diag.cu -- population diversity: the pairwise Hamming distance between
// replica configurations, corrected for the global spin-flip symmetry of
// Max-Cut, d_H = min(d, n - d) (Suppl., Hamming distance of replicas).
//
// The +-1 spins are packed one bit per spin (a warp ballot per 32 spins of a
// row), then every pair r < r' is counted by XOR and popcount over the packed
// words, tile by tile: a CTA owns a 32 x 32 block of pairs and stages 32 words
// of both row sets in shared memory per round.  Results are exact integers:
// a histogram over the corrected distance and its sum.
#include "pamc_device.cuh"
#include "pamc_internal.h"

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

}  // namespace

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
