// schedule.cu -- the shared random sweep order of Sec. III.A ("all spins were
// sequentially updated once in a randomized order"), turned into dependency
// levels for a parallel sweep with exactly sequential semantics.
//
// The order of (t, sweep) sorts the vertices by the 32-bit key
// Philox(k, sweep, t, PERM<<24)[0], ties by index.  Only the relative order of
// coupled vertices matters for a sequential single-spin sweep: the decision at
// vertex k reads the fields of k, which only its neighbours change.  So vertex
// k is placed at level 1 + max(level of neighbours that come before k), and
// all vertices of one level (pairwise uncoupled) can be updated at once,
// level after level, giving bit-identical results to the sequential order.
// Levels are produced by Kahn's algorithm, frontier by frontier; no sort is
// needed.  One CTA builds one (t, sweep) schedule; a launch builds the
// schedules of several steps at once.  The keys and predecessor counters sit
// in shared memory when 8n bytes fit (global scratch otherwise), and a
// frontier narrower than the CTA gives each vertex several lanes, which split
// its neighbour list.
#include <algorithm>

#include "pamc_device.cuh"
#include "pamc_internal.h"

namespace pamc {

namespace {

__device__ __forceinline__ bool before(uint32_t ka, int32_t a, uint32_t kb, int32_t b) {
    return ka < kb || (ka == kb && a < b);
}

constexpr int kSchedThreads = 512;
constexpr size_t kSchedSmemMax = 160 * 1024;   // keys and counters of n <= 20,480 in shared memory

__device__ __forceinline__ void
schedule_body(int32_t n, const int32_t *__restrict__ rp, const uint32_t *__restrict__ adj,
              uint32_t key0, uint32_t key1, int32_t t0, int32_t S, int32_t slots,
              int32_t *__restrict__ order, int32_t *__restrict__ lvl_ptr, int32_t *__restrict__ nlev,
              uint32_t *__restrict__ skey, int32_t *__restrict__ scnt, uint32_t *__restrict__ ell,
              int32_t W, int2 *__restrict__ pos, int b, size_t smem_bytes) {
    extern __shared__ uint32_t ssched[];
    const int ti = b / S, sw = b % S;
    const int32_t t = t0 + ti;
    const int slot = t % slots;
    const size_t base = (size_t)slot * S + sw;
    int32_t *ord = order + base * (size_t)n;
    int32_t *lp = lvl_ptr + base * (size_t)(n + 1);
    const bool in_smem = (size_t)n * 8 <= smem_bytes;
    uint32_t *key = in_smem ? ssched : skey + (size_t)b * n;
    int32_t *cnt = in_smem ? reinterpret_cast<int32_t *>(ssched + n) : scnt + (size_t)b * n;
    __shared__ int32_t s_tail;
    __shared__ int32_t s_end;

    for (int32_t k = threadIdx.x; k < n; k += blockDim.x)
        key[k] = philox((uint32_t)k, (uint32_t)sw, (uint32_t)t, kTagPerm << 24, key0, key1).x;
    if (threadIdx.x == 0) s_tail = 0;
    __syncthreads();

    // number of coupled predecessors; sources form level 0
    for (int32_t k = threadIdx.x; k < n; k += blockDim.x) {
        const uint32_t kk = key[k];
        int32_t c = 0;
        for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
            const int32_t j = (int32_t)(adj[e] & 0xFFFFFFu);
            c += before(key[j], j, kk, k) ? 1 : 0;
        }
        cnt[k] = c;
        if (c == 0) ord[atomicAdd(&s_tail, 1)] = k;
    }
    __syncthreads();
    int32_t beg = 0, end = s_tail;
    int32_t L = 0;
    if (threadIdx.x == 0) lp[0] = 0;
    while (beg < end) {
        if (threadIdx.x == 0) lp[L + 1] = end;
        // lanes per frontier vertex: the largest power of two up to 32 that
        // still leaves a lane group for every vertex of the frontier
        int lpv = 1;
        while (lpv < 32 && (int32_t)(blockDim.x / (2 * lpv)) >= end - beg) lpv *= 2;
        const int32_t sub = threadIdx.x % lpv, step = blockDim.x / lpv;
        for (int32_t i = beg + threadIdx.x / lpv; i < end; i += step) {
            const int32_t k = ord[i];
            const uint32_t kk = key[k];
            for (int32_t e = rp[k] + sub; e < rp[k + 1]; e += lpv) {
                const int32_t j = (int32_t)(adj[e] & 0xFFFFFFu);
                if (before(kk, k, key[j], j) && atomicSub(&cnt[j], 1) == 1)
                    ord[atomicAdd(&s_tail, 1)] = j;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_end = s_tail;
        __syncthreads();
        beg = end;
        end = s_end;
        ++L;
    }
    if (threadIdx.x == 0) nlev[base] = L;
    __syncthreads();
    // Within a level the order is free (its vertices are uncoupled), so each
    // level is grouped by degree (counting sort into eight classes, stable
    // enough for the purpose): the lanes of a warp then walk rows of similar
    // length in the sweep.  The counters' array is free now and holds the
    // sorted copy.
    {
        __shared__ int32_t bc[8];
        int32_t *tmp = cnt;
        auto dclass = [&](int32_t k) {
            const int32_t d = rp[k + 1] - rp[k];
            return d <= 4 ? 0 : d <= 8 ? 1 : d <= 12 ? 2 : d <= 16 ? 3 : d <= 24 ? 4 : d <= 32 ? 5 : d <= 64 ? 6 : 7;
        };
        for (int32_t l = 0; l < L; ++l) {
            const int32_t b0 = lp[l], b1 = lp[l + 1];
            if (b1 - b0 < 64) continue;   // one or two warps: nothing to gain
            if (threadIdx.x < 8) bc[threadIdx.x] = 0;
            __syncthreads();
            for (int32_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&bc[dclass(ord[i])], 1);
            __syncthreads();
            if (threadIdx.x == 0) {
                int32_t acc = b0;
                for (int c = 0; c < 8; ++c) { const int32_t v = bc[c]; bc[c] = acc; acc += v; }
            }
            __syncthreads();
            for (int32_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
                const int32_t k = ord[i];
                tmp[atomicAdd(&bc[dclass(k)], 1)] = k;
            }
            __syncthreads();
            for (int32_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) ord[i] = tmp[i];
            __syncthreads();
        }
    }
    // Position-indexed neighbour lists: order[i] becomes k | deg << 24 (deg =
    // nonzero couplings).  With an ELL buffer (width W, a multiple of 4) the
    // couplings of position i go to ell[(i/32)*32*W + s*32 + i%32], s < deg,
    // and the slots deg..W-1 hold 0 (vertex 0, coupling 0), so that a warp's
    // lanes read consecutive words, the first four slots can be read before
    // deg is known, and pos[i] = {k | deg << 24, sum_j J_kj}.
    uint32_t *es = ell ? ell + base * (size_t)(((n + 31) >> 5) << 5) * W : nullptr;
    int2 *ps = pos ? pos + base * (size_t)n : nullptr;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int32_t k = ord[i];
        int32_t d = 0, jsum = 0;
        uint32_t *ep = es ? es + (size_t)(i >> 5) * 32 * W + (i & 31) : nullptr;
        for (int32_t e = rp[k]; e < rp[k + 1]; ++e) {
            const uint32_t a = adj[e];
            const int32_t J = (int32_t)a >> 24;
            if (J == 0) continue;
            if (ep) ep[(size_t)d * 32] = a;
            ++d;
            jsum += J;
        }
        if (ep)
            for (int32_t s2 = d; s2 < W; ++s2) ep[(size_t)s2 * 32] = 0u;
        ord[i] = k | (d << 24);
        if (ps) ps[i] = make_int2(k | (d << 24), jsum);
    }
}

__global__ void __launch_bounds__(kSchedThreads)
k_schedule(int32_t n, const int32_t *__restrict__ rp, const uint32_t *__restrict__ adj,
           uint32_t key0, uint32_t key1, int32_t t0, int32_t S, int32_t slots,
           int32_t *__restrict__ order, int32_t *__restrict__ lvl_ptr, int32_t *__restrict__ nlev,
           uint32_t *__restrict__ skey, int32_t *__restrict__ scnt, uint32_t *__restrict__ ell,
           int32_t W, int2 *__restrict__ pos, size_t smem_bytes) {
    schedule_body(n, rp, adj, key0, key1, t0, S, slots, order, lvl_ptr, nlev, skey, scnt, ell, W, pos,
                  blockIdx.x, smem_bytes);
}

__global__ void __launch_bounds__(kSchedThreads)
k_schedule_batched(const SchedDesc *__restrict__ descs, const int2 *__restrict__ items, size_t smem_bytes) {
    const int2 it = items[blockIdx.x];
    const SchedDesc d = descs[it.x];
    int32_t t0 = d.t0;
    if (d.ctl) {
        if (d.ctl->done) return;
        t0 = d.ctl->t + d.ahead;
        if (t0 >= d.t_end) return;
    }
    schedule_body(d.n, d.rp, d.adj, d.key0, d.key1, t0, d.S, d.slots, d.order, d.lvl, d.nlev, d.skey,
                  d.scnt, d.ell, d.W, d.pos, it.y, smem_bytes);
}

}  // namespace

void launch_schedule(int32_t n, const int32_t *rp, const uint32_t *adj, uint64_t seed, int32_t t0,
                     int32_t nt, int32_t S, int32_t /*slot0*/, int32_t slots, int32_t *order,
                     int32_t *lvl_ptr, int32_t *nlev, uint32_t *skey, int32_t *scnt,
                     cudaStream_t st, uint32_t *ell, int32_t W, int2 *pos) {
    if (nt <= 0 || S <= 0) return;
    size_t smem = (size_t)n * 8 <= kSchedSmemMax ? (size_t)n * 8 : 0;
    if (allow_dynamic_smem(k_schedule, smem) != cudaSuccess) smem = 0;   // the global-scratch path
    k_schedule<<<nt * S, kSchedThreads, smem, st>>>(n, rp, adj, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                     t0, S, slots, order, lvl_ptr, nlev, skey, scnt,
                                                     ell, W, pos, smem);
}

void launch_schedule_batched(const SchedDesc *descs, const int2 *items, int32_t nitems, int32_t n_max,
                             cudaStream_t st) {
    if (nitems <= 0) return;
    // members whose 8n bytes exceed this use their global scratch
    size_t smem = std::min((size_t)n_max * 8, kSchedSmemMax);
    if (allow_dynamic_smem(k_schedule_batched, smem) != cudaSuccess) smem = 0;   // the global-scratch path
    k_schedule_batched<<<nitems, kSchedThreads, smem, st>>>(descs, items, smem);
}

}  // namespace pamc
