// noalloc.cu -- pamc_sweeps_noalloc: S single-spin sweeps of an Ising
// population at a fixed beta, for callers that cannot allocate device memory
// (code running where cudaMalloc is forbidden or unavailable: inside a host
// framework that owns all device memory, a real-time loop, or a plug-in that
// may only use the buffers it is handed).  The call uses the same schedule,
// table and sweep kernels as pamc_step; everything those kernels need beyond
// the caller's inputs and outputs lives in one file-scope device array of
// fixed size, reserved when the library is loaded and held by every GPU that
// loads it until the process exits.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "pamc_internal.h"

namespace pamc {
cudaError_t launch_tables(int kind, int rule, int32_t H, const DevCtl *ctl, uint64_t *tab,
                          cudaStream_t st);
}

using namespace pamc;

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the static scratch (offsets in bytes, each 256-byte aligned).
constexpr size_t kOffCtl = 0;
constexpr size_t kOffTab = kOffCtl + align256(sizeof(DevCtl));
constexpr size_t kOffAdj = kOffTab + align256(sizeof(uint64_t) * 255);
constexpr size_t kOffParent = kOffAdj + align256(sizeof(uint32_t) * PAMC_NOALLOC_MAX_NNZ);
constexpr size_t kOffNcm = kOffParent + align256(sizeof(int32_t) * PAMC_NOALLOC_MAX_R);
constexpr size_t kOffOrder = kOffNcm + align256(sizeof(int32_t) * PAMC_NOALLOC_MAX_R);
constexpr size_t kOffLvl = kOffOrder +
    align256(sizeof(int32_t) * (size_t)PAMC_NOALLOC_MAX_SWEEPS * PAMC_NOALLOC_MAX_N);
constexpr size_t kOffNlev = kOffLvl +
    align256(sizeof(int32_t) * (size_t)PAMC_NOALLOC_MAX_SWEEPS * (PAMC_NOALLOC_MAX_N + 1));
constexpr size_t kOffKey = kOffNlev + align256(sizeof(int32_t) * PAMC_NOALLOC_MAX_SWEEPS);
constexpr size_t kOffCnt = kOffKey +
    align256(sizeof(uint32_t) * (size_t)PAMC_NOALLOC_MAX_SWEEPS * PAMC_NOALLOC_MAX_N);
constexpr size_t kScratchBytes = kOffCnt +
    align256(sizeof(int32_t) * (size_t)PAMC_NOALLOC_MAX_SWEEPS * PAMC_NOALLOC_MAX_N);
static_assert(kScratchBytes == PAMC_NOALLOC_SCRATCH_BYTES,
              "PAMC_NOALLOC_SCRATCH_BYTES in pamc.h must match the scratch layout");

// The scratch.  In host code this name is only a stand-in: the device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_base[kMaxDevices] = {};

void set_msg(char *err, size_t len, const char *fmt, ...) {
    if (!err || len == 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, len, fmt, ap);
    va_end(ap);
}

// Reset the parts of the scratch that must start fresh on every call.
__global__ void k_noalloc_reset(DevCtl *ctl, double beta, int32_t *parent, int32_t *ncm_idx,
                                int32_t R) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->done = 0;
        ctl->err = 0;
        ctl->beta = beta;
    }
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        parent[r] = r;      // no resampling: slot r reads replica r
        ncm_idx[r] = -1;    // no cluster move
    }
}

// Validate the caller's device CSR and pack it as (col | (-w) << 24).
// Symmetry as a multiset: (j, w) occurs in row i exactly as often as (i, w)
// in row j (the schedule counts a vertex's earlier neighbours over its own
// row and counts them down over theirs, so an unmatched duplicate would leave
// a vertex unscheduled); |w| <= 127; no self loop; every row's sum |w| <= H.
// Errors set ctl->err (first error wins).
__global__ void k_noalloc_pack(int32_t n, int32_t nnz, const int32_t *__restrict__ rp,
                               const int32_t *__restrict__ col, const int32_t *__restrict__ w,
                               int32_t H, uint32_t *__restrict__ adj, DevCtl *ctl) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t b = rp[i], e1 = rp[i + 1];
        if (b < 0 || (i == 0 && b != 0) || e1 < b || e1 > nnz || (i == n - 1 && e1 != nnz)) {
            atomicCAS(&ctl->err, 0, (int)PAMC_ERR_ARG);
            continue;
        }
        int32_t habs = 0;
        for (int32_t e = b; e < e1; ++e) {
            const int32_t j = col[e], we = w[e];
            if (j < 0 || j >= n) { atomicCAS(&ctl->err, 0, (int)PAMC_ERR_ARG); break; }
            if (j == i) { atomicCAS(&ctl->err, 0, (int)PAMC_ERR_DIAG); break; }
            if (we < -127 || we > 127) { atomicCAS(&ctl->err, 0, (int)PAMC_ERR_RANGE); break; }
            habs += we < 0 ? -we : we;
            const int32_t jb = rp[j], je = rp[j + 1];
            int32_t fwd = 0, bwd = 0;
            for (int32_t f = b; f < e1; ++f) fwd += (col[f] == j && w[f] == we) ? 1 : 0;
            if (jb >= 0 && je <= nnz && jb <= je)
                for (int32_t f = jb; f < je; ++f) bwd += (col[f] == i && w[f] == we) ? 1 : 0;
            if (fwd != bwd) { atomicCAS(&ctl->err, 0, (int)PAMC_ERR_ASYM); break; }
            adj[e] = (uint32_t)j | ((uint32_t)(uint8_t)(int8_t)(-we) << 24);
        }
        if (habs > H) atomicCAS(&ctl->err, 0, (int)PAMC_ERR_RANGE);
    }
}

unsigned char *scratch_base(int dev, char *err, size_t len, pamc_status &st) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices) {
        st = PAMC_ERR_ARG;
        set_msg(err, len, "device index %d out of range", dev);
        return nullptr;
    }
    if (!g_base[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            st = PAMC_ERR_CUDA;
            set_msg(err, len, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return nullptr;
        }
        g_base[dev] = static_cast<unsigned char *>(p);
    }
    st = PAMC_OK;
    return g_base[dev];
}

}  // namespace

extern "C" pamc_status pamc_sweeps_noalloc(int32_t n, int32_t nnz, const int32_t *row_ptr,
                                           const int32_t *col, const int32_t *w, int32_t H,
                                           int32_t rule, int32_t R, int32_t sweeps, double beta,
                                           uint64_t seed, int32_t t, const int8_t *spins_in,
                                           int8_t *spins_out, int64_t *E_out, void *stream,
                                           char *err, size_t err_len) {
    set_msg(err, err_len, "%s", "");
    if (n < 1 || n > PAMC_NOALLOC_MAX_N) {
        set_msg(err, err_len, "n = %d outside [1, %d]", n, PAMC_NOALLOC_MAX_N);
        return PAMC_ERR_RANGE;
    }
    if (nnz < 0 || nnz > PAMC_NOALLOC_MAX_NNZ) {
        set_msg(err, err_len, "nnz = %d outside [0, %d]", nnz, PAMC_NOALLOC_MAX_NNZ);
        return PAMC_ERR_RANGE;
    }
    if (sweeps < 0 || sweeps > PAMC_NOALLOC_MAX_SWEEPS) {
        set_msg(err, err_len, "sweeps = %d outside [0, %d]", sweeps, PAMC_NOALLOC_MAX_SWEEPS);
        return PAMC_ERR_RANGE;
    }
    if (R < 1 || R > PAMC_NOALLOC_MAX_R) {
        set_msg(err, err_len, "R = %d outside [1, %d]", R, PAMC_NOALLOC_MAX_R);
        return PAMC_ERR_RANGE;
    }
    if (H < 0 || H > 127) {
        set_msg(err, err_len, "H = %d outside [0, 127]", H);
        return PAMC_ERR_RANGE;
    }
    if (rule != 0 && rule != 1) {
        set_msg(err, err_len, "rule must be 0 (heat-bath) or 1 (Metropolis)");
        return PAMC_ERR_ARG;
    }
    if (!row_ptr || (nnz > 0 && (!col || !w)) || !spins_in || !spins_out || !E_out ||
        !(beta == beta) || t < 0) {
        set_msg(err, err_len, "null pointer, NaN beta or negative t");
        return PAMC_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_msg(err, err_len, "cudaGetDevice: %s", cudaGetErrorString(e));
        return PAMC_ERR_CUDA;
    }
    pamc_status st;
    unsigned char *base = scratch_base(dev, err, err_len, st);
    if (!base) return st;
    cudaStream_t s = (cudaStream_t)stream;
    DevCtl *ctl = reinterpret_cast<DevCtl *>(base + kOffCtl);
    uint64_t *tab = reinterpret_cast<uint64_t *>(base + kOffTab);
    uint32_t *adj = reinterpret_cast<uint32_t *>(base + kOffAdj);
    int32_t *parent = reinterpret_cast<int32_t *>(base + kOffParent);
    int32_t *ncm_idx = reinterpret_cast<int32_t *>(base + kOffNcm);
    int32_t *order = reinterpret_cast<int32_t *>(base + kOffOrder);
    int32_t *lvl = reinterpret_cast<int32_t *>(base + kOffLvl);
    int32_t *nlev = reinterpret_cast<int32_t *>(base + kOffNlev);
    uint32_t *skey = reinterpret_cast<uint32_t *>(base + kOffKey);
    int32_t *scnt = reinterpret_cast<int32_t *>(base + kOffCnt);

    k_noalloc_reset<<<(R + 255) / 256, 256, 0, s>>>(ctl, beta, parent, ncm_idx, R);
    k_noalloc_pack<<<(n + 255) / 256, 256, 0, s>>>(n, nnz, row_ptr, col, w, H, adj, ctl);
    // the instance must be valid before any kernel indexes through it
    int32_t derr = 0;
    e = cudaMemcpyAsync(&derr, &ctl->err, sizeof(derr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_msg(err, err_len, "validation: %s", cudaGetErrorString(e));
        return PAMC_ERR_CUDA;
    }
    if (derr != 0) {
        set_msg(err, err_len, "invalid instance (status %d)", derr);
        return (pamc_status)derr;
    }
    pamc_params p{};
    p.kind = 0;
    p.rule = rule;
    p.R = R;
    p.sweeps = sweeps;
    p.seed = seed;
    if (sweeps > 0)
        launch_schedule(n, row_ptr, adj, seed, t, 1, sweeps, 0, 1, order, lvl, nlev, skey, scnt, s);
    e = launch_tables(0, rule, H, ctl, tab, s);
    SweepCfg cfg{1, n >= 16384 ? 8 : n >= 4096 ? 4 : n >= 1024 ? 2 : 1};
    // spins_in may equal spins_out: the sweep's CTA for a replica group reads
    // the group's rows completely into shared memory before its first write,
    // and no other CTA touches those rows
    if (e == cudaSuccess)
        e = launch_sweep(0, rule, n, row_ptr, adj, H, p, t, 0, SchedView{order, lvl, nlev, nullptr, nullptr, 0}, tab,
                         spins_in, parent, nullptr, ncm_idx, spins_out, E_out, ctl, cfg, 0, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&derr, &ctl->err, sizeof(derr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_msg(err, err_len, "sweeps: %s", cudaGetErrorString(e));
        return PAMC_ERR_CUDA;
    }
    if (derr != 0) {
        set_msg(err, err_len, "device reported status %d", derr);
        return (pamc_status)derr;
    }
    return PAMC_OK;
}
