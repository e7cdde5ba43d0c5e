// shard.cu -- one population split over several processes (one GPU each):
// the host-side exchange plan of a step and the kernel that gathers the
// replica rows a process sends.
//
// The resampling of Eq. 1-2 is global over the R replicas: the new slot m
// copies the old replica parent[m], wherever it lives.  Slots are split in
// equal contiguous blocks (process q owns slots [q c, (q + 1) c), c = R /
// nranks, a multiple of 4 so that no group of four replicas straddles two
// processes).  Every process computes the same parent map from the gathered
// energies, so every process can work out, without further messages, which
// of its old replicas each other process needs and where the ones it
// receives will sit.  Systematic resampling gives a nondecreasing parent
// map, so most parents are local and only the replicas near a block's edges
// move; the plan does not rely on that.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "pamc_internal.h"

namespace pamc {

namespace {

// One CTA per row; 16-byte words when the row length and both pointers allow.
__global__ void k_gather_rows(int32_t n, const int32_t *__restrict__ rows, int32_t nrows,
                              const int8_t *__restrict__ src, int8_t *__restrict__ dst, int vec) {
    for (int32_t i = blockIdx.x; i < nrows; i += gridDim.x) {
        const int8_t *s = src + (size_t)rows[i] * n;
        int8_t *d = dst + (size_t)i * n;
        if (vec) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(s);
            uint4 *d4 = reinterpret_cast<uint4 *>(d);
            for (int32_t k = threadIdx.x; k < n / 16; k += blockDim.x) d4[k] = s4[k];
        } else {
            for (int32_t k = threadIdx.x; k < n; k += blockDim.x) d[k] = s[k];
        }
    }
}

}  // namespace

cudaError_t launch_gather_rows(int32_t n, const int32_t *rows, int32_t nrows, const int8_t *src, int8_t *dst,
                               cudaStream_t st) {
    if (nrows <= 0) return cudaSuccess;
    const int vec = (n % 16 == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0) &&
                    ((reinterpret_cast<uintptr_t>(dst) & 15) == 0);
    const int grid = std::min<int32_t>(nrows, 152 * 8);
    k_gather_rows<<<grid, 256, 0, st>>>(n, rows, nrows, src, dst, vec);
    return cudaGetLastError();
}

}  // namespace pamc

extern "C" pamc_status pamc_shard_range(int32_t R, int32_t nranks, int32_t rank, int32_t *base, int32_t *count) {
    if (!base || !count || nranks < 1 || rank < 0 || rank >= nranks || R < 1 || R % (4 * nranks) != 0)
        return PAMC_ERR_ARG;
    *count = R / nranks;
    *base = rank * *count;
    return PAMC_OK;
}

extern "C" pamc_status pamc_shard_plan(int32_t R, int32_t nranks, int32_t rank, const int32_t *parent,
                                       int32_t *send_counts, int32_t *send_rows, int32_t *recv_counts,
                                       int32_t *local_parent) {
    int32_t base = 0, c = 0;
    if (pamc_shard_range(R, nranks, rank, &base, &c) != PAMC_OK) return PAMC_ERR_ARG;
    if (!parent || !send_counts || !send_rows || !recv_counts || !local_parent) return PAMC_ERR_ARG;
    for (int32_t m = 0; m < R; ++m)
        if (parent[m] < 0 || parent[m] >= R) return PAMC_ERR_RANGE;
    // receive side: the distinct foreign parents of the own slots, ordered by
    // global index (which orders them by owner too); they follow the own
    // rows in the sweep's source buffer
    std::vector<char> need(R, 0);
    for (int32_t m = 0; m < c; ++m) {
        const int32_t p = parent[base + m];
        if (p / c != rank) need[p] = 1;
    }
    std::vector<int32_t> row_of(R, -1);
    std::fill(recv_counts, recv_counts + nranks, 0);
    int32_t next = c;
    for (int32_t p = 0; p < R; ++p)
        if (need[p]) {
            row_of[p] = next++;
            recv_counts[p / c] += 1;
        }
    for (int32_t m = 0; m < c; ++m) {
        const int32_t p = parent[base + m];
        local_parent[m] = p / c == rank ? p - base : row_of[p];
    }
    // send side: for every other process, the distinct own replicas that
    // are parents of its slots, in the same (global index) order
    std::vector<char> mark(c);
    int32_t ns = 0;
    for (int32_t q = 0; q < nranks; ++q) {
        send_counts[q] = 0;
        if (q == rank) continue;
        std::fill(mark.begin(), mark.end(), 0);
        for (int32_t m = q * c; m < (q + 1) * c; ++m) {
            const int32_t p = parent[m];
            if (p / c == rank) mark[p - base] = 1;
        }
        for (int32_t j = 0; j < c; ++j)
            if (mark[j]) {
                send_rows[ns++] = j;
                send_counts[q] += 1;
            }
    }
    return PAMC_OK;
}
