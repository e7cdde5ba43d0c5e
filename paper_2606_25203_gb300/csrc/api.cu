// api.cu -- the C ABI of libpamc (declared in include/pamc.h): instance
// validation and upload, device memory of a run, and the per-iteration launch
// sequence of Algorithm 1.  Host code only marshals arguments and enqueues
// kernels; every step of an iteration runs on the GPU, and the controller
// state stays in device memory so the host never waits inside a run.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pamc_internal.h"

// NVTX ranges around the host-side phases (a profiler shows the kernels each
// phase enqueued under its name; without a tool attached a range is a
// pointer check)
namespace {
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace
#define PAMC_CAT2(a, b) a##b
#define PAMC_CAT(a, b) PAMC_CAT2(a, b)
#define PAMC_RANGE(name) NvtxRange PAMC_CAT(pamc_range_, __LINE__)(name)

using namespace pamc;

namespace pamc {
cudaError_t launch_tables(int kind, int rule, int32_t H, const DevCtl *ctl, uint64_t *tab,
                          cudaStream_t st);
cudaError_t launch_prep(const pamc_params &p, const int64_t *E_src, DevCtl *ctl, int32_t *parent,
                        int32_t *count, int32_t *ncm_idx, int32_t *targets, int32_t *fam, uint64_t *qbuf,
                        cudaStream_t st, long long *mm = nullptr);
cudaError_t launch_ncm(int32_t n, const int32_t *rp, const uint32_t *adj, const pamc_params &p,
                       const int8_t *src, const int64_t *E_src, const int32_t *parent,
                       const int32_t *targets, int8_t *ncm_buf, uint32_t *nkey,
                       DevCtl *ctl, cudaStream_t st, int32_t base = 0, int32_t count = -1,
                       const int32_t *prow = nullptr);
cudaError_t launch_control(int32_t n, int64_t W, const pamc_params &p, const int64_t *E,
                           const int8_t *spins, int8_t *best, DevCtl *ctl, cudaStream_t st,
                           int32_t base = 0, int32_t count = -1);
size_t prep_smem_bytes(int32_t R);
}  // namespace pamc

namespace {

pamc_alloc_fn g_alloc = nullptr;
pamc_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
thread_local char g_create_err[256] = "";

constexpr int kSchedSlots = 16;   // schedules of this many steps are built per launch
constexpr size_t kSmemMax = 227 * 1024;   // opt-in shared memory per CTA

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct pamc_handle_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t n = 0, nnz = 0, H = 0;
    int32_t maxdeg = 0;        // largest number of nonzero couplings of a vertex
    int32_t ell_w = 0;         // ELL width of the schedules (0: CSR reads)
    int64_t W = 0;
    int dense = 0;
    // instance
    int32_t *d_rp = nullptr;
    uint32_t *d_adj = nullptr;
    int4 *d_nibc = nullptr;      // per-vertex constants of the biased 4-bit lanes, or nullptr
    // run
    pamc_params p{};
    int initialized = 0;
    int64_t host_t = 0;
    // Algorithm 1's iteration counter z as the controller will hold it at
    // the start of step host_t (1 after init, z + 1 each step, back to 1
    // after the restart at z = z_rst): the host launches a restart's re-draw
    // only in the step that restarts
    int32_t host_z = 1;
    int64_t sched_end = 0;     // schedules exist for steps < sched_end
    SweepCfg cfg{1, 1};
    std::vector<DevBuf> bufs;  // every device allocation of the run
    std::vector<DevBuf> inst_bufs;
    int8_t *d_spins[2] = {nullptr, nullptr};
    int64_t *d_E[2] = {nullptr, nullptr};
    int32_t *d_parent = nullptr, *d_count = nullptr, *d_ncm_idx = nullptr, *d_targets = nullptr;
    uint64_t *d_q = nullptr;   // resampling weights (sparse handles)
    long long *d_mm = nullptr; // E_min / E_max of a large population (R > kPrepOneCtaMaxR)
    int32_t *d_fam = nullptr;   // [2][R] lineage (family of each slot)
    int8_t *d_ncm_buf = nullptr;
    uint32_t *d_nkey = nullptr;
    uint64_t *d_tab = nullptr;
    int32_t *d_order = nullptr, *d_lvl = nullptr, *d_nlev = nullptr, *d_scnt = nullptr;
    uint32_t *d_skey = nullptr;
    uint32_t *d_ell = nullptr;
    int2 *d_pos = nullptr;
    uint32_t *d_gsp = nullptr;   // Ising: replica groups' spin words in device memory
    bool gsp = false;            // the single-run sweeps use d_gsp (groups that do not fit on chip)
    bool nib = false;            // the single-run sweeps use 4-bit lanes, eight replicas a word
    DevCtl *d_ctl = nullptr;
    int8_t *d_best = nullptr;
    // dense instances
    int8_t *d_J = nullptr;               // n x n couplings (J = -w)
    int32_t *d_H = nullptr;              // [R][n] fields
    uint8_t *d_Sb = nullptr;             // [64][n] e4m3 population for the tcgen05 recompute
    bool dense_tc = false;               // recompute on tcgen05 (n a multiple of 16)
    bool dense_tcu = false;              // field update of the sweep on tcgen05
    alignas(64) unsigned char tm_J[128];  // tensor maps of J and of d_Sb
    alignas(64) unsigned char tm_S[128];
    int32_t *d_perm = nullptr, *d_sidx = nullptr, *d_G = nullptr, *d_ident = nullptr, *d_nonc = nullptr;
    int32_t *d_boff = nullptr;           // bucket offsets of the order sort
    uint32_t *d_pkey = nullptr;
    uint32_t *d_T = nullptr, *d_T2 = nullptr;   // bit tiles of the dense chains
    unsigned long long *d_flip = nullptr, *d_snew = nullptr;
    void *d_bar = nullptr;
    int32_t dense_Hc = 0, dense_grid = 0, dense_nupd = 0, dense_rows = 0;
    int32_t dense_R = 0;                 // replicas this handle sweeps (p.R unless split over processes)
    int64_t launches = 0;
    // device time of the sweep launches (pamc_set_sweep_timing): events
    // recorded on the handle's stream around each sweep launch, in pairs
    bool time_sweeps = false;
    std::vector<cudaEvent_t> sweep_ev;
    size_t sweep_ev_used = 0;      // pairs recorded and not yet folded
    double sweep_ms = 0.0;         // time of the pairs folded since the last read
    int64_t sweep_timed = 0;       // sweep launches timed since the last read
    // a population split over processes (pamc_shard_init): this handle owns
    // slots [sh_base, sh_base + sh_count) of the p.R replicas; the energies,
    // parent map, counts and controller cover all p.R, the spins only its own
    // slots and, during a step, the foreign parents it received
    bool sharded = false;
    int32_t sh_rank = 0, sh_nranks = 1, sh_base = 0, sh_count = 0;
    int sh_phase = 0;              // next call: 0 resample, 1 sweep, 2 control
    int32_t *d_plocal = nullptr;   // [sh_count] source row of each own slot's parent
    int32_t *d_rows = nullptr;     // [p.R] own rows to send
    uint64_t inst_hash = 0;        // FNV-1a of the packed CSR (0 for dense instances)
    char err[256] = "";
};

namespace {

pamc_status fail(pamc_handle h, pamc_status s, const char *fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) snprintf(h->err, sizeof(h->err), "%s", buf);
    else snprintf(g_create_err, sizeof(g_create_err), "%s", buf);
    return s;
}

pamc_status cuda_fail(pamc_handle h, cudaError_t e, const char *what) {
    return fail(h, PAMC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *dev_alloc(pamc_handle h, size_t bytes, std::vector<DevBuf> &list) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (g_alloc) {
        p = g_alloc(bytes, h->device, (void *)h->stream, g_alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) list.push_back({p, bytes});
    return p;
}

void dev_free_all(pamc_handle h, std::vector<DevBuf> &list) {
    if (!list.empty()) cudaStreamSynchronize(h->stream);
    for (auto &b : list) {
        if (g_free) g_free(b.p, h->device, (void *)h->stream, g_alloc_ctx);
        else cudaFree(b.p);
    }
    list.clear();
}

template <typename T>
bool alloc_n(pamc_handle h, T *&ptr, size_t count, std::vector<DevBuf> &list) {
    ptr = static_cast<T *>(dev_alloc(h, count * sizeof(T), list));
    return ptr != nullptr;
}

// Validated symmetric CSR -> packed adjacency (col | J<<24 with J = -w).
pamc_status validate_csr(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                         std::vector<uint32_t> &adj, int64_t &W, int32_t &H, int32_t &maxdeg) {
    if (n < 1 || n >= (1 << 24) || !rp || (!col && rp && rp[n] > 0) || (!w && rp && rp[n] > 0))
        return fail(nullptr, PAMC_ERR_ARG, "invalid n or null CSR pointer");
    if (rp[0] != 0) return fail(nullptr, PAMC_ERR_ARG, "row_ptr[0] must be 0");
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return fail(nullptr, PAMC_ERR_ARG, "row_ptr not monotone at %d", i);
    const int32_t nnz = rp[n];
    std::vector<std::tuple<int32_t, int32_t, int32_t>> fwd, bwd;
    fwd.reserve(nnz);
    bwd.reserve(nnz);
    adj.resize(nnz);
    W = 0;
    H = 0;
    maxdeg = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t habs = 0;
        int32_t deg = 0;
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = col[e];
            if (j < 0 || j >= n) return fail(nullptr, PAMC_ERR_ARG, "column index out of range");
            if (j == i) return fail(nullptr, PAMC_ERR_DIAG, "self loop at vertex %d", i);
            if (w[e] < -127 || w[e] > 127)
                return fail(nullptr, PAMC_ERR_RANGE, "|w| > 127 at (%d,%d)", i, j);
            fwd.emplace_back(i, j, w[e]);
            bwd.emplace_back(j, i, w[e]);
            habs += w[e] < 0 ? -w[e] : w[e];
            deg += w[e] != 0 ? 1 : 0;
            W += w[e];
            const int32_t J = -w[e];
            adj[e] = (uint32_t)j | ((uint32_t)(uint8_t)(int8_t)J << 24);
        }
        if (habs > kWideLaneMaxH)
            return fail(nullptr, PAMC_ERR_RANGE, "sum_j |w_ij| = %lld > %d at vertex %d",
                        (long long)habs, kWideLaneMaxH, i);
        H = std::max<int32_t>(H, (int32_t)habs);
        maxdeg = std::max(maxdeg, deg);
    }
    std::sort(fwd.begin(), fwd.end());
    std::sort(bwd.begin(), bwd.end());
    if (fwd != bwd) return fail(nullptr, PAMC_ERR_ASYM, "coupling matrix is not symmetric");
    W /= 2;
    return PAMC_OK;
}

// Sum the recorded pairs into sweep_ms (waits for the stream).
cudaError_t fold_sweep_events(pamc_handle h) {
    if (h->sweep_ev_used == 0) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    for (size_t i = 0; e == cudaSuccess && i < h->sweep_ev_used; ++i) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->sweep_ev[2 * i], h->sweep_ev[2 * i + 1]);
        h->sweep_ms += ms;
    }
    h->sweep_ev_used = 0;
    return e;
}

// Events around one sweep launch when timing is on; at most 1024 pairs are
// kept before they are folded (a wait for the stream every 1024 launches).
cudaError_t sweep_timer(pamc_handle h, bool after) {
    if (!h->time_sweeps) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!after) {
        if (h->sweep_ev_used == 1024) e = fold_sweep_events(h);
        while (e == cudaSuccess && h->sweep_ev.size() < 2 * (h->sweep_ev_used + 1)) {
            cudaEvent_t ev;
            e = cudaEventCreate(&ev);
            if (e == cudaSuccess) h->sweep_ev.push_back(ev);
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->sweep_ev[2 * h->sweep_ev_used], h->stream);
    } else {
        e = cudaEventRecord(h->sweep_ev[2 * h->sweep_ev_used + 1], h->stream);
        h->sweep_ev_used += 1;
        h->sweep_timed += 1;
    }
    return e;
}

void release_run(pamc_handle h) {
    dev_free_all(h, h->bufs);
    h->initialized = 0;
    h->d_spins[0] = h->d_spins[1] = nullptr;
    h->d_gsp = nullptr;
    h->gsp = false;
    h->nib = false;
    h->sharded = false;
    h->sh_rank = 0; h->sh_nranks = 1; h->sh_base = 0; h->sh_count = 0; h->sh_phase = 0;
    h->d_plocal = h->d_rows = nullptr;
    h->d_mm = nullptr;
}

// The controller restarts at the end of a step that begins with z >= z_rst;
// advance the host's copy of z past one step.
bool restart_due(const pamc_handle_s *h) {
    return h->p.z_rst > 0 && h->p.restart_reinit && h->host_z >= h->p.z_rst;
}
void advance_z(pamc_handle_s *h) { h->host_z = (h->p.z_rst > 0 && h->host_z >= h->p.z_rst) ? 1 : h->host_z + 1; }

// Words of the replica groups' spins in device memory (n_pad per group).
size_t gsp_words(int32_t n, int32_t R) { return (size_t)((R + 3) / 4) * (size_t)((n + 3) & ~3); }

// Launch shape of the sweep kernel: groups per CTA, warps per group and
// lanes per vertex.  Ising runs on ELL schedules give each group a CTA of its
// own, sized for the latency of a level, unless the SMs are shared and the
// levels are too wide for more than one lane per vertex; Potts runs do the
// same (one lane per vertex) where an average level fits the group's share
// of the SM in one pass.  Otherwise every (gpc, wpg) is scored by the fraction of group slots used
// over whole waves, the lane efficiency of a level (average level size over
// the lanes of a group), and resident warps per SM; Ising runs on ELL
// schedules then give the lanes a level leaves idle to the couplings (the
// largest power of two up to 8 at which an average level still fits the
// group's lanes in one pass).  PAMC_SWEEP_CFG="gpc,wpg[,lpv]" overrides.
int sweep_kind(const pamc_params &p) { return p.kind == 0 ? 0 : (p.rule == 2 ? 2 : 1); }

SweepCfg choose_cfg(int kind, int32_t n, int32_t R, int32_t H, double avg_level, double avg_deg, int sms,
                    int32_t ell_w) {
    const int32_t groups = (R + 3) / 4;   // every sweep kind groups four replicas
    const bool lpv_ok = kind == 0 && ell_w > 4;
    if (const char *env = getenv("PAMC_SWEEP_CFG")) {
        int a = 0, b = 0, v = 1;
        const int got = sscanf(env, "%d,%d,%d", &a, &b, &v);
        if (got >= 2 && a >= 1 && a <= 15 && b >= 1 && a * b * 32 <= 1024 &&
            v >= 1 && v <= 32 && (v & (v - 1)) == 0) {
            // Ising: lanes per vertex on ELL rows; the cascaded Potts sweep:
            // lane pairs (2) on ELL rows; the softmax Potts sweep: quads (4)
            const int lpv = lpv_ok ? v : (kind == 1 && ell_w > 0 && v == 2) ? 2 : (kind == 2 && v == 4) ? 4 : 1;
            SweepCfg c{a, b, lpv};
            if (sweep_smem_bytes(kind, n, H, c) <= 227 * 1024) return c;
        }
    }
    if (kind == 0 && ell_w > 0) {
        // Groups sized for the latency of a level: lanes per vertex so that
        // the eight slots a lane loads ahead cover an average row (half that
        // where four or more groups share an SM, and two groups to a CTA
        // there), halved while an average level needs more lanes than a
        // group's share of the SM (1024 threads over the groups an SM
        // holds), then warps so that an average level takes one pass.
        // Where that leaves one lane per vertex on a shared SM, the scoring
        // below decides.
        const int64_t per_sm = (groups + sms - 1) / std::max(sms, 1);
        int lanes = 1024;
        while (lanes > 32 && (int64_t)lanes * per_sm > 1024) lanes >>= 1;
        const double lev = std::max(avg_level, 1.0);
        SweepCfg c{per_sm >= 4 ? 2 : 1, 1, 1};
        if (lpv_ok)
            while (c.lanes_per_vertex < 32 && 8.0 * c.lanes_per_vertex < avg_deg) c.lanes_per_vertex *= 2;
        if (per_sm >= 4 && c.lanes_per_vertex > 1) c.lanes_per_vertex >>= 1;
        while (c.lanes_per_vertex > 1 && lev * c.lanes_per_vertex > lanes) c.lanes_per_vertex >>= 1;
        while (c.warps_per_group * 32 < lanes && 32.0 * c.warps_per_group < lev * c.lanes_per_vertex)
            c.warps_per_group *= 2;
        if ((per_sm <= 1 || c.lanes_per_vertex > 1) && sweep_smem_bytes(kind, n, H, c) <= 227 * 1024) return c;
    }
    if (kind != 0) {
        // Potts: one group per CTA with warps for one pass over an average
        // level, where that fits the group's share of the SM; wide levels or
        // crowded SMs take the scoring below
        const int64_t per_sm = (groups + sms - 1) / std::max(sms, 1);
        int lanes = 1024;
        while (lanes > 32 && (int64_t)lanes * per_sm > 1024) lanes >>= 1;
        SweepCfg c{1, 1, 1};
        while (c.warps_per_group < 32 && 32.0 * c.warps_per_group < std::max(avg_level, 1.0)) c.warps_per_group *= 2;
        if (32 * c.warps_per_group <= lanes && sweep_smem_bytes(kind, n, H, c) <= 227 * 1024) {
            // several lanes a position -- the cascaded sampler on ELL rows:
            // pairs; the softmax sampler: quads -- with twice the warps where
            // that still fits the group's share of the SM, two groups to a
            // CTA where the SMs hold two or more (configuration 3: cascaded
            // 0.720 against 0.773 ms per step, softmax 1.65 against 2.08, for
            // one group of four warps a CTA, one lane a position)
            if (((kind == 1 && ell_w > 0) || kind == 2) && c.warps_per_group <= 16 &&
                64 * c.warps_per_group <= lanes) {
                SweepCfg p2{1, 2 * c.warps_per_group, kind == 2 ? 4 : 2};
                if (groups >= 2 * (int64_t)sms && 2 * 32 * p2.warps_per_group <= 1024) p2.groups_per_cta = 2;
                if (sweep_smem_bytes(kind, n, H, p2) <= 227 * 1024) return p2;
            }
            return c;
        }
    }
    SweepCfg best{1, 1};
    double best_score = -1.0;
    for (int wpg = 1; wpg <= 16; wpg *= 2) {
        const int tpg = wpg * 32;
        const double iters = std::ceil(std::max(avg_level, 1.0) / tpg);
        const double lane_eff = std::max(avg_level, 1.0) / (iters * tpg);
        for (int gpc = 1; gpc <= 15 && gpc * tpg <= 1024; ++gpc) {
            const SweepCfg c{gpc, wpg};
            const size_t smem = sweep_smem_bytes(kind, n, H, c);
            if (smem > 227 * 1024) break;
            const int threads = gpc * tpg;
            const int bps = std::min({2048 / threads, (int)(233472 / (smem + 1024)),
                                      65536 / (64 * threads)});
            if (bps < 1) continue;
            const int64_t ctas = (groups + gpc - 1) / gpc;
            const int64_t slots = (int64_t)sms * bps;
            const int64_t waves = (ctas + slots - 1) / slots;
            const double util = (double)groups / ((double)waves * slots * gpc);
            const double warps = (double)std::min<int64_t>(ctas, slots) / sms * gpc * wpg;
            const double occ = std::min(1.0, warps / 32.0);
            const double score = util * lane_eff * (0.5 + 0.5 * occ);
            if (score > best_score + 1e-9) { best_score = score; best = c; }
        }
    }
    if (lpv_ok) {
        const double lev = std::ceil(std::max(avg_level, 1.0));
        const int tpg = best.warps_per_group * 32;
        while (best.lanes_per_vertex < 8 && lev * best.lanes_per_vertex * 2 <= tpg &&
               4 * best.lanes_per_vertex < ell_w)
            best.lanes_per_vertex *= 2;
    }
    return best;
}

// ---------------------------------------------------------------- dense runs
// H = J S for the population given by (src, parent, ncm_idx)
cudaError_t dense_recompute(pamc_handle h, const int8_t *src, const int32_t *parent, const int32_t *ncm_idx,
                            int restart_t) {
    if (h->dense_tc)
        return launch_dense_recompute_tc(h->n, h->dense_R, h->tm_J, h->tm_S, src, parent, nullptr, ncm_idx, h->d_Sb,
                                         h->d_H, h->d_ctl, h->stream, restart_t);
    return launch_dense_recompute(h->n, h->dense_R, h->d_J, src, parent, nullptr, ncm_idx, h->d_H, h->d_ctl,
                                  h->stream, restart_t);
}

// own: the replicas this handle sweeps (base: the first one's index in the
// whole population of p.R); own = p.R unless the population is split.
pamc_status init_dense(pamc_handle h, pamc_params p, int32_t base, int32_t own, bool split) {
    if (p.kind != 0) return fail(h, PAMC_ERR_ARG, "dense instances run the Ising (Max-Cut) kind only");
    if (own > 64) return fail(h, PAMC_ERR_RANGE, "dense instances support at most 64 replicas per handle");
    if (p.R > kPrepOneCtaMaxR) return fail(h, PAMC_ERR_RANGE, "dense populations hold at most %d replicas",
                                            kPrepOneCtaMaxR);
    if (p.stagnation && (h->n & 1))
        return fail(h, PAMC_ERR_ARG, "cluster moves on dense instances need even n (no iso-sites then)");
    if (p.sweeps > 64) return fail(h, PAMC_ERR_RANGE, "dense instances support at most 64 sweeps per step");
    int coop = 0, sms = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (!coop) return fail(h, PAMC_ERR_CUDA, "device lacks cooperative launch");
    const int32_t n = h->n, R = own, Rg = p.R, S = std::max(p.sweeps, 1);
    const int chain = (R + 3) / 4;
    const int grid = sms;
    const int nupd = grid - chain;
    if (nupd < 1) return fail(h, PAMC_ERR_RANGE, "too few SMs for the dense sweep");
    // field update on the tensor cores (fields in tensor memory) when n allows TMA-style rows
    const char *sw_env = getenv("PAMC_DENSE_UPDATE");   // "cuda": the CUDA-core update
    const bool tcu = dense_tc_supported(n) && !(sw_env && strcmp(sw_env, "cuda") == 0);
    int32_t rows = (n + nupd - 1) / nupd;
    if (tcu) rows = (rows + 31) & ~31;
    const size_t smem = dense_sweep_smem(n, R, rows, tcu);
    if (rows > dense_sweep_threads() || smem > 227 * 1024)
        return fail(h, PAMC_ERR_RANGE, "dense instance too large for the on-chip field slices");
    release_run(h);
    h->p = p;
    h->dense_grid = grid;
    h->dense_nupd = nupd;
    h->dense_rows = rows;
    h->dense_tcu = tcu;
    h->dense_Hc = std::min<int32_t>(n, 32767);
    h->dense_R = R;
    const int B = dense_block_positions();
    const size_t tabn = (size_t)2 * h->dense_Hc + 1;
    // spin rows: the own replicas, and as many again for received parents
    const size_t rows_sp = split ? 2 * (size_t)R : (size_t)R;
    bool ok = alloc_n(h, h->d_spins[0], rows_sp * n, h->bufs) &&
              alloc_n(h, h->d_spins[1], rows_sp * n, h->bufs) &&
              alloc_n(h, h->d_E[0], 64, h->bufs) && alloc_n(h, h->d_E[1], 64, h->bufs) &&
              alloc_n(h, h->d_parent, Rg, h->bufs) && alloc_n(h, h->d_count, Rg, h->bufs) &&
              alloc_n(h, h->d_fam, 2 * (size_t)Rg, h->bufs) &&
              alloc_n(h, h->d_ncm_idx, Rg, h->bufs) && alloc_n(h, h->d_targets, Rg, h->bufs) &&
              alloc_n(h, h->d_tab, tabn, h->bufs) && alloc_n(h, h->d_ctl, 1, h->bufs) &&
              alloc_n(h, h->d_best, n, h->bufs) && alloc_n(h, h->d_H, (size_t)R * n, h->bufs) &&
              alloc_n(h, h->d_perm, (size_t)S * n, h->bufs) && alloc_n(h, h->d_pkey, (size_t)S * n, h->bufs) &&
              alloc_n(h, h->d_sidx, (size_t)S * n, h->bufs) && alloc_n(h, h->d_G, (size_t)2 * B * 64, h->bufs) &&
              alloc_n(h, h->d_T, (size_t)2 * B * (B / 32), h->bufs) && alloc_n(h, h->d_T2, (size_t)2 * B * (B / 32), h->bufs) &&
              alloc_n(h, h->d_flip, (size_t)3 * B, h->bufs) && alloc_n(h, h->d_snew, (size_t)3 * B, h->bufs) &&
              (h->d_bar = dev_alloc(h, 64, h->bufs)) != nullptr &&
              alloc_n(h, h->d_ident, R, h->bufs) && alloc_n(h, h->d_nonc, R, h->bufs) &&
              alloc_n(h, h->d_boff, dense_perm_offsets(S), h->bufs);
    if (ok && split) ok = alloc_n(h, h->d_plocal, R, h->bufs) && alloc_n(h, h->d_rows, Rg, h->bufs);
    const char *rc_env = getenv("PAMC_DENSE_RECOMPUTE");   // "mma": the mma.sync kernel
    h->dense_tc = dense_tc_supported(n) && !(rc_env && strcmp(rc_env, "mma") == 0);
    if (ok && h->dense_tc) {
        ok = alloc_n(h, h->d_Sb, (size_t)64 * n, h->bufs);
        if (ok && (dense_tc_map(h->tm_J, h->d_J, n, n, 256) != cudaSuccess ||
                   dense_tc_map(h->tm_S, h->d_Sb, 64, n, 64) != cudaSuccess))
            h->dense_tc = false;
    }
    if (!ok) {
        release_run(h);
        return fail(h, PAMC_ERR_OOM, "device allocation of the dense population failed");
    }
    DevCtl c;
    memset(&c, 0, sizeof(c));
    c.z = 1;
    c.beta = p.beta0;
    c.dbeta = p.steps > 1 ? (p.beta1 - p.beta0) / (double)(p.steps - 1) : 0.0;
    c.delta = c.dbeta;
    c.mstar = INT64_MIN;
    c.best_replica = -1;
    std::vector<int32_t> ident(Rg), ones(Rg, 1), minus(Rg, -1);
    for (int32_t r = 0; r < Rg; ++r) ident[r] = r;
    cudaError_t e = cudaMemcpyAsync(h->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_parent, ident.data(), 4 * Rg, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_fam, ident.data(), 4 * Rg, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_ident, ident.data(), 4 * R, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_count, ones.data(), 4 * Rg, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_ncm_idx, minus.data(), 4 * Rg, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_nonc, minus.data(), 4 * R, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_best, 0, n, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_E[0], 0, 64 * 8, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_E[1], 0, 64 * 8, h->stream);
    // initial population, its fields (tensor-core recompute) and energies
    if (e == cudaSuccess)
        e = launch_init_spins(0, 0, n, R, p.seed, 0, 0, h->d_ctl, h->d_spins[0], h->stream, base);
    if (e == cudaSuccess)
        e = dense_recompute(h, h->d_spins[0], h->d_ident, h->d_nonc, -1);
    if (e == cudaSuccess)
        e = launch_dense_energy(n, R, h->d_H, h->d_spins[0], h->d_E[0], h->d_ctl, h->stream, -1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "dense init");
    h->launches += 3;
    h->host_t = 0;
    h->host_z = 1;
    h->initialized = 1;
    return PAMC_OK;
}

pamc_status step_dense(pamc_handle h, int32_t nsteps) {
    PAMC_RANGE("pamc_step (dense)");
    const pamc_params &p = h->p;
    const int32_t n = h->n, R = p.R;
    pamc_params pp = p;
    pp.n_top = 0;   // no cluster-move targets: dense moves are provably empty for even n
    for (int32_t i = 0; i < nsteps; ++i) {
        const int64_t t = h->host_t;
        if (t > INT32_MAX - 2) return fail(h, PAMC_ERR_RANGE, "step counter overflow");
        int8_t *src = h->d_spins[t & 1], *dst = h->d_spins[(t + 1) & 1];
        int64_t *Es = h->d_E[t & 1], *Ed = h->d_E[(t + 1) & 1];
        cudaError_t e = launch_dense_perm(n, p.seed, (int32_t)t, p.sweeps, h->d_perm, h->d_pkey, h->d_sidx,
                                          h->d_boff, h->d_ctl, h->stream);
        if (e == cudaSuccess)
            e = launch_prep(pp, Es, h->d_ctl, h->d_parent, h->d_count, h->d_ncm_idx, h->d_targets, h->d_fam,
                            nullptr, h->stream);
        if (e == cudaSuccess) e = launch_dense_tables(p.rule, h->dense_Hc, n, h->d_ctl, h->d_tab, h->stream);
        if (e == cudaSuccess)
            e = dense_recompute(h, src, h->d_parent, h->d_ncm_idx, -1);
        if (e == cudaSuccess) e = sweep_timer(h, false);
        if (e == cudaSuccess)
            e = launch_dense_sweep(n, R, p.sweeps, p.rule, h->dense_Hc, (int32_t)t, p.seed, h->dense_nupd,
                                   h->dense_rows, h->dense_grid, h->d_J, h->d_perm, h->d_tab, src,
                                   h->d_parent, nullptr, h->d_ncm_idx, h->d_H, dst, Ed, h->d_G, h->d_T,
                                   h->d_T2, h->d_flip, h->d_snew, h->d_bar, h->d_ctl, h->stream, h->dense_tcu);
        if (e == cudaSuccess) e = sweep_timer(h, true);
        if (e == cudaSuccess) e = launch_control(n, h->W, p, Ed, dst, h->d_best, h->d_ctl, h->stream);
        h->launches += 7;
        if (e == cudaSuccess && restart_due(h)) {
            const int32_t tk = (int32_t)(t + 1);
            e = launch_init_spins(0, 0, n, R, p.seed, tk, 1, h->d_ctl, dst, h->stream);
            if (e == cudaSuccess)
                e = dense_recompute(h, dst, h->d_ident, h->d_nonc, tk);
            if (e == cudaSuccess) e = launch_dense_energy(n, R, h->d_H, dst, Ed, h->d_ctl, h->stream, tk);
            h->launches += 3;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "dense kernel launch");
        h->host_t = t + 1;
        advance_z(h);
    }
    return PAMC_OK;
}

}  // namespace

extern "C" {

pamc_status pamc_set_allocator(pamc_alloc_fn alloc, pamc_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(nullptr, PAMC_ERR_ARG, "allocator and free function must both be set or both NULL");
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return PAMC_OK;
}

pamc_status pamc_create_csr(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            const int32_t *w, int cuda_device, void *stream, pamc_handle *out) {
    if (!out) return fail(nullptr, PAMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::vector<uint32_t> adj;
    int64_t W = 0;
    int32_t H = 0, maxdeg = 0;
    pamc_status s = validate_csr(n, row_ptr, col, w, adj, W, H, maxdeg);
    if (s != PAMC_OK) return s;
    cudaError_t e = cudaSetDevice(cuda_device);
    if (e != cudaSuccess) return fail(nullptr, PAMC_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    pamc_handle h = new (std::nothrow) pamc_handle_s();
    if (!h) return fail(nullptr, PAMC_ERR_OOM, "host allocation failed");
    h->device = cuda_device;
    h->stream = (cudaStream_t)stream;
    h->n = n;
    h->nnz = row_ptr[n];
    h->W = W;
    h->H = H;
    h->maxdeg = maxdeg;
    {   // identifies the instance in checkpoints (pamc_save / pamc_load)
        uint64_t x = 1469598103934665603ull;
        auto mix = [&x](uint32_t v) {
            for (int b = 0; b < 4; ++b) { x ^= (v >> (8 * b)) & 0xFFu; x *= 1099511628211ull; }
        };
        for (int32_t i = 0; i <= n; ++i) mix((uint32_t)row_ptr[i]);
        for (uint32_t a : adj) mix(a);
        h->inst_hash = x;
    }
    // position-indexed ELL when its padding stays within 4x the couplings
    // (the schedule's position record holds the degree in 8 bits)
    const int64_t ell_entries = (int64_t)((n + 31) / 32) * 32 * ((maxdeg + 3) & ~3);
    h->ell_w = (maxdeg > 0 && maxdeg < 256 && ell_entries <= 4 * (int64_t)h->nnz + 4096) ? ((maxdeg + 3) & ~3) : 0;
    // field ranges beyond the fixed 4-bit bias (7) but within 15 a half-row:
    // the biased 4-bit lanes' per-vertex constants
    std::vector<int4> nibc;
    const bool biased = h->ell_w > 0 && !(H <= kNibbleMaxH && (h->ell_w == 4 || h->ell_w == 8)) &&
                        nibble_biased_constants(n, row_ptr, adj.data(), H, h->ell_w, nibc);
    if (!alloc_n(h, h->d_rp, (size_t)n + 1, h->inst_bufs) ||
        !alloc_n(h, h->d_adj, (size_t)std::max(h->nnz, 1), h->inst_bufs) ||
        (biased && !alloc_n(h, h->d_nibc, (size_t)n, h->inst_bufs))) {
        dev_free_all(h, h->inst_bufs);
        delete h;
        return fail(nullptr, PAMC_ERR_OOM, "device allocation of the instance failed");
    }
    e = cudaMemcpyAsync(h->d_rp, row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && h->nnz > 0)
        e = cudaMemcpyAsync(h->d_adj, adj.data(), sizeof(uint32_t) * h->nnz, cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess && biased)
        e = cudaMemcpyAsync(h->d_nibc, nibc.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        dev_free_all(h, h->inst_bufs);
        delete h;
        return fail(nullptr, PAMC_ERR_CUDA, "instance upload: %s", cudaGetErrorString(e));
    }
    *out = h;
    return PAMC_OK;
}

pamc_status pamc_create_dense(int32_t n, const int8_t *w, int w_on_device, int cuda_device,
                              void *stream, pamc_handle *out) {
    if (!out) return fail(nullptr, PAMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 2 || !w) return fail(nullptr, PAMC_ERR_ARG, "n >= 2 and a weight matrix are required");
    if ((int64_t)n > (int64_t)1 << 20) return fail(nullptr, PAMC_ERR_RANGE, "n > 2^20");
    cudaError_t e = cudaSetDevice(cuda_device);
    if (e != cudaSuccess) return fail(nullptr, PAMC_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    pamc_handle h = new (std::nothrow) pamc_handle_s();
    if (!h) return fail(nullptr, PAMC_ERR_OOM, "host allocation failed");
    h->device = cuda_device;
    h->stream = (cudaStream_t)stream;
    h->n = n;
    h->dense = 1;
    h->nnz = 0;
    h->H = 0;
    const size_t total = (size_t)n * n;
    unsigned long long *d_sum = nullptr;
    int *d_err = nullptr;
    if (!alloc_n(h, h->d_J, total, h->inst_bufs) || !alloc_n(h, d_sum, 1, h->inst_bufs) ||
        !alloc_n(h, d_err, 1, h->inst_bufs)) {
        dev_free_all(h, h->inst_bufs);
        delete h;
        return fail(nullptr, PAMC_ERR_OOM, "device allocation of the dense instance failed");
    }
    e = cudaMemcpyAsync(h->d_J, w, total, w_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_sum, 0, sizeof(*d_sum), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(*d_err), h->stream);
    if (e == cudaSuccess) e = launch_dense_negate_sum(total, h->d_J, d_sum, h->stream);
    if (e == cudaSuccess) e = launch_dense_validate(n, h->d_J, d_err, h->stream);
    if (e == cudaSuccess) e = launch_dense_to_e4m3(total, h->d_J, h->stream);   // stored as e4m3 bytes
    unsigned long long wsum = 0;
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&wsum, d_sum, sizeof(wsum), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof(err), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->launches += 2;
    if (e != cudaSuccess || err != 0) {
        dev_free_all(h, h->inst_bufs);
        delete h;
        if (e != cudaSuccess) return fail(nullptr, PAMC_ERR_CUDA, "dense upload: %s", cudaGetErrorString(e));
        return fail(nullptr, (pamc_status)err, "dense matrix rejected: %s",
                    err == PAMC_ERR_ASYM ? "not symmetric" : err == PAMC_ERR_DIAG ? "nonzero diagonal"
                                                                            : "entries must be +-1 off the diagonal");
    }
    h->W = (int64_t)wsum / 2;   // sum over ordered pairs counts each edge twice
    *out = h;
    return PAMC_OK;
}

// nranks = 0: the whole population on this handle (pamc_init); else this
// handle's share of a population split over nranks processes.
static pamc_status init_run(pamc_handle h, const pamc_params *pp, int32_t rank, int32_t nranks) {
    if (!h || !pp) return fail(h, PAMC_ERR_ARG, "null handle or params");
    PAMC_RANGE("pamc_init");
    pamc_params p = *pp;
    if (p.K == 0) p.K = 3;
    if (p.kind != 0 && p.kind != 1) return fail(h, PAMC_ERR_ARG, "kind must be 0 or 1");

    if (p.kind == 0 && p.rule != 0 && p.rule != 1) return fail(h, PAMC_ERR_ARG, "Ising rule must be 0 or 1");
    if (p.kind == 1 && !((p.rule == 0 && p.K == 3) || (p.rule == 2 && p.K >= 2 && p.K <= 8)))
        return fail(h, PAMC_ERR_ARG, "Potts: rule 0 (cascaded) needs K = 3, rule 2 (softmax) 2 <= K <= 8");
    if (p.kind == 1 && p.rule == 2 && !(p.gamma >= 0.0 && p.gamma < 1e30))
        return fail(h, PAMC_ERR_ARG, "softmax noise amplitude gamma must be finite and >= 0");
    if (p.R < 1 || p.R > kMaxPopulation) return fail(h, PAMC_ERR_RANGE, "R must be in [1, %d]", kMaxPopulation);
    if (p.sweeps < 0 || p.steps < 1) return fail(h, PAMC_ERR_ARG, "sweeps >= 0 and steps >= 1 required");
    if (p.win_short < 0 || p.win_long < 0 || p.win_short > kHistMax || p.win_long > kHistMax)
        return fail(h, PAMC_ERR_RANGE, "stagnation windows must be in [0, %d]", kHistMax);
    if (p.n_top <= 0) p.n_top = std::max(1, p.R / 16);
    if (p.R > kPrepOneCtaMaxR && p.stagnation && p.kind == 0 && std::min(p.n_top, p.R) > kNcmSelectMaxTop)
        return fail(h, PAMC_ERR_RANGE, "populations above %d take at most %d NCM targets (n_top)", kPrepOneCtaMaxR,
                    kNcmSelectMaxTop);
    if (p.mis_trials < 0) return fail(h, PAMC_ERR_ARG, "mis_trials must be >= 0");
    if (!(p.beta0 == p.beta0) || !(p.beta1 == p.beta1)) return fail(h, PAMC_ERR_ARG, "beta is NaN");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    int32_t base = 0, own = p.R;   // own slots [base, base + own)
    if (nranks > 0 && pamc_shard_range(p.R, nranks, rank, &base, &own) != PAMC_OK)
        return fail(h, PAMC_ERR_ARG, "split population: need 0 <= rank < nranks and R a multiple of 4 nranks");
    if (h->dense) {
        const pamc_status s = init_dense(h, p, base, own, nranks > 0);
        if (s == PAMC_OK && nranks > 0) {
            h->sharded = true;
            h->sh_rank = rank;
            h->sh_nranks = nranks;
            h->sh_base = base;
            h->sh_count = own;
            h->sh_phase = 0;
        }
        return s;
    }
    if (p.kind == 1 && h->H > kByteLaneMaxH)
        return fail(h, PAMC_ERR_RANGE, "Max-3-Cut runs need sum_j |w_ij| <= %d (this instance: %d)", kByteLaneMaxH,
                    h->H);
    release_run(h);
    h->p = p;
    const int32_t n = h->n, R = p.R, S = std::max(p.sweeps, 1);
    const int32_t ntop = std::min(p.n_top, R);
    const size_t tabn = p.kind == 0 ? (size_t)(2 * h->H + 1)
                                    : (size_t)(4 * h->H + 1) * (4 * h->H + 1) + (4 * h->H + 1);
    // spin rows: the own slots, and as many again for received parents
    const size_t rows = nranks > 0 ? 2 * (size_t)own : (size_t)R;
    bool ok = alloc_n(h, h->d_spins[0], rows * n, h->bufs) &&
              alloc_n(h, h->d_spins[1], rows * n, h->bufs) &&
              alloc_n(h, h->d_E[0], own, h->bufs) && alloc_n(h, h->d_E[1], own, h->bufs) &&
              alloc_n(h, h->d_q, R, h->bufs) &&
              alloc_n(h, h->d_parent, R, h->bufs) && alloc_n(h, h->d_count, R, h->bufs) &&
              alloc_n(h, h->d_fam, 2 * (size_t)R, h->bufs) &&
              alloc_n(h, h->d_ncm_idx, R, h->bufs) && alloc_n(h, h->d_targets, R, h->bufs) &&
              alloc_n(h, h->d_tab, tabn, h->bufs) && alloc_n(h, h->d_ctl, 1, h->bufs) &&
              alloc_n(h, h->d_best, n, h->bufs) &&
              alloc_n(h, h->d_order, (size_t)kSchedSlots * S * n, h->bufs) &&
              alloc_n(h, h->d_lvl, (size_t)kSchedSlots * S * (n + 1), h->bufs) &&
              alloc_n(h, h->d_nlev, (size_t)kSchedSlots * S, h->bufs) &&
              alloc_n(h, h->d_skey, (size_t)kSchedSlots * S * n, h->bufs) &&
              alloc_n(h, h->d_scnt, (size_t)kSchedSlots * S * n, h->bufs);
    if (ok && h->ell_w > 0) {
        ok = alloc_n(h, h->d_ell, (size_t)kSchedSlots * S * ((n + 31) / 32) * 32 * h->ell_w, h->bufs) &&
             alloc_n(h, h->d_pos, (size_t)kSchedSlots * S * n, h->bufs);
    } else {
        h->d_ell = nullptr;
        h->d_pos = nullptr;
    }
    if (ok && p.stagnation && p.kind == 0)
        ok = alloc_n(h, h->d_ncm_buf, (size_t)ntop * n, h->bufs) &&
             alloc_n(h, h->d_nkey, (size_t)ntop * n, h->bufs);
    if (ok && nranks > 0) ok = alloc_n(h, h->d_plocal, own, h->bufs) && alloc_n(h, h->d_rows, R, h->bufs);
    if (ok && R > kPrepOneCtaMaxR) ok = alloc_n(h, h->d_mm, 2, h->bufs);
    if (!ok) {
        release_run(h);
        return fail(h, PAMC_ERR_OOM, "device allocation of the population failed");
    }
    DevCtl c;
    memset(&c, 0, sizeof(c));
    c.t = 0;
    c.z = 1;
    c.beta = p.beta0;
    c.dbeta = p.steps > 1 ? (p.beta1 - p.beta0) / (double)(p.steps - 1) : 0.0;
    c.delta = c.dbeta;
    c.mstar = INT64_MIN;
    c.best_replica = -1;
    e = cudaMemcpyAsync(h->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "controller upload");
    std::vector<int32_t> ident(R), ones(R, 1), minus(R, -1);
    for (int32_t r = 0; r < R; ++r) ident[r] = r;
    e = cudaMemcpyAsync(h->d_parent, ident.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_fam, ident.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_count, ones.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_ncm_idx, minus.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_best, 0, n, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "initial state upload");
    e = launch_init(p.kind, p.K, n, h->d_rp, h->d_adj, own, p.seed, 0, 0, h->d_ctl, h->W, h->d_spins[0],
                    h->d_E[0], h->stream, base);
    if (e != cudaSuccess) return cuda_fail(h, e, "initial population");
    h->launches += 2;
    // host copies of the host-side vectors must stay alive until the copies ran
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "init");
    // schedules of the first steps; their depth sets the sweep launch shape
    double avg_level = n;
    h->sched_end = 0;
    if (p.sweeps > 0) {
        launch_schedule(n, h->d_rp, h->d_adj, p.seed, 0, kSchedSlots, p.sweeps, 0, kSchedSlots,
                        h->d_order, h->d_lvl, h->d_nlev, h->d_skey, h->d_scnt, h->stream, h->d_ell,
                        h->ell_w, h->d_pos);
        h->launches += 1;
        h->sched_end = kSchedSlots;
        int32_t depth = 0;
        e = cudaMemcpyAsync(&depth, h->d_nlev, sizeof(depth), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "schedule depth readback");
        avg_level = (double)n / std::max(depth, 1);
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    h->cfg = choose_cfg(sweep_kind(p), n, own, h->H, avg_level, (double)h->nnz / std::max(n, 1), sms, h->ell_w);
    // Ising groups whose spin words do not fit shared memory (or all of them
    // with PAMC_SWEEP_GLOBAL=1) keep the words in device memory: one lane per
    // vertex, one group per CTA
    const char *genv = getenv("PAMC_SWEEP_GLOBAL");
    const bool wide = p.kind == 0 && h->H > kByteLaneMaxH;   // 16-bit field lanes, one lane per vertex
    if (wide) h->cfg.lanes_per_vertex = 1;
    if (p.kind == 0 && ((genv && genv[0] == '1') || sweep_smem_bytes(0, n, h->H, h->cfg) > kSmemMax)) {
        if (!getenv("PAMC_SWEEP_CFG")) h->cfg = SweepCfg{1, 16, 1};
        h->cfg.lanes_per_vertex = 1;
        if (!alloc_n(h, h->d_gsp, gsp_words(n, own) * (wide ? 2 : 1), h->bufs)) {
            release_run(h);
            return fail(h, PAMC_ERR_OOM, "device allocation of the group spin words failed");
        }
        h->gsp = true;
    }
    // field ranges of at most 7 on ELL rows of width 4 or 8, or of 15 a
    // half-row on rows up to 16 wide: eight replicas a word (groups of eight,
    // shaped like a population of half the size)
    if (p.kind == 0 && !h->gsp && sweep_nibble_ok(h->H, p.sweeps, h->ell_w, 1, false, h->d_nibc != nullptr) &&
        !sweep_push_enabled()) {
        SweepCfg c = choose_cfg(0, n, 4 * ((own + 7) / 8), h->H, avg_level, (double)h->nnz / std::max(n, 1), sms,
                                h->ell_w);
        c.lanes_per_vertex = 1;
        // a one-group CTA keeps at least one pass of its warps busy per
        // average level (down to 8 warps): with less, a lane has no next
        // position whose loads could overlap the current one
        if (!getenv("PAMC_SWEEP_CFG"))
            while (c.groups_per_cta == 1 && c.warps_per_group > 8 && avg_level < 32.0 * c.warps_per_group)
                c.warps_per_group >>= 1;
        if (sweep_nibble_smem_bytes(n, h->H, c) <= kSmemMax) {
            h->cfg = c;
            h->nib = true;
        }
    }
    if (!h->gsp && sweep_smem_bytes(sweep_kind(p), n, h->H, h->cfg) > kSmemMax) {
        release_run(h);
        return fail(h, PAMC_ERR_RANGE, "n = %d: one replica group's labels exceed shared memory", n);
    }
    h->host_t = 0;
    h->host_z = 1;
    if (nranks > 0) {
        h->sharded = true;
        h->sh_rank = rank;
        h->sh_nranks = nranks;
        h->sh_base = base;
        h->sh_count = own;
        h->sh_phase = 0;
    }
    h->initialized = 1;
    return PAMC_OK;
}

pamc_status pamc_init(pamc_handle h, const pamc_params *pp) { return init_run(h, pp, 0, 0); }

pamc_status pamc_shard_init(pamc_handle h, const pamc_params *p, int32_t rank, int32_t nranks) {
    if (nranks < 1) return fail(h, PAMC_ERR_ARG, "nranks must be >= 1");
    return init_run(h, p, rank, nranks);
}

pamc_status pamc_step(pamc_handle h, int32_t nsteps) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_step before pamc_init");
    if (h->sharded) return fail(h, PAMC_ERR_STATE, "a split population steps through the pamc_shard_* calls");
    if (nsteps < 0) return fail(h, PAMC_ERR_ARG, "nsteps < 0");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (h->dense) return step_dense(h, nsteps);
    PAMC_RANGE("pamc_step");
    const pamc_params &p = h->p;
    const int32_t n = h->n;
    for (int32_t i = 0; i < nsteps; ++i) {
        PAMC_RANGE("iteration");
        const int64_t t = h->host_t;
        if (t > INT32_MAX - 2) return fail(h, PAMC_ERR_RANGE, "step counter overflow");
        if (p.sweeps > 0 && t >= h->sched_end) {
            launch_schedule(n, h->d_rp, h->d_adj, p.seed, (int32_t)t, kSchedSlots, p.sweeps, 0,
                            kSchedSlots, h->d_order, h->d_lvl, h->d_nlev, h->d_skey, h->d_scnt,
                            h->stream, h->d_ell, h->ell_w, h->d_pos);
            h->sched_end = t + kSchedSlots;
            h->launches += 1;
        }
        int8_t *src = h->d_spins[t & 1], *dst = h->d_spins[(t + 1) & 1];
        int64_t *Es = h->d_E[t & 1], *Ed = h->d_E[(t + 1) & 1];
        e = launch_prep(p, Es, h->d_ctl, h->d_parent, h->d_count, h->d_ncm_idx, h->d_targets, h->d_fam,
                        h->d_q, h->stream, h->d_mm);
        if (e == cudaSuccess) e = launch_tables(p.kind, p.rule, h->H, h->d_ctl, h->d_tab, h->stream);
        h->launches += 3;
        if (e == cudaSuccess && p.stagnation && p.kind == 0) {
            e = launch_ncm(n, h->d_rp, h->d_adj, p, src, Es, h->d_parent, h->d_targets, h->d_ncm_buf,
                           h->d_nkey, h->d_ctl, h->stream);
            h->launches += 1;
        }
        SchedView sv{h->d_order, h->d_lvl, h->d_nlev, h->d_ell, h->d_pos, h->ell_w, h->d_nibc};
        if (e == cudaSuccess) e = sweep_timer(h, false);
        if (e == cudaSuccess)
            e = launch_sweep(sweep_kind(p), p.rule, n, h->d_rp, h->d_adj, h->H, p, (int32_t)t,
                             (int32_t)(t % kSchedSlots), sv, h->d_tab, src, h->d_parent,
                             h->d_ncm_buf, h->d_ncm_idx, dst, Ed, h->d_ctl, h->cfg, h->W, h->stream,
                             h->gsp ? h->d_gsp : nullptr, 0, h->nib);
        if (e == cudaSuccess) e = sweep_timer(h, true);
        if (e == cudaSuccess) e = launch_control(n, h->W, p, Ed, dst, h->d_best, h->d_ctl, h->stream);
        h->launches += 2;
        if (e == cudaSuccess && restart_due(h)) {
            e = launch_init(p.kind, p.K, n, h->d_rp, h->d_adj, p.R, p.seed, (int32_t)(t + 1), 1, h->d_ctl,
                            h->W, dst, Ed, h->stream);
            h->launches += 2;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
        h->host_t = t + 1;
        advance_z(h);
    }
    return PAMC_OK;
}

pamc_status pamc_sync(pamc_handle h) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    if (h->initialized) {
        int32_t err = 0;
        e = cudaMemcpy(&err, (const char *)h->d_ctl + offsetof(DevCtl, err), sizeof(err),
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "error flag readback");
        if (err != 0) return fail(h, (pamc_status)err, "device reported error %d", err);
    }
    return PAMC_OK;
}

// ---------------------------------------------------------------- split population
// One iteration of Algorithm 1 in three calls, with the caller's exchange
// between them (the calls of pamc_step, in the same order and with the same
// random streams; every process runs the population step and the controller
// on all R energies and so takes the same decisions).

static pamc_status read_ctl(pamc_handle h, DevCtl &c);

static pamc_status shard_check(pamc_handle h, int phase, const char *what) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    if (!h->initialized || !h->sharded) return fail(h, PAMC_ERR_STATE, "%s: no split population initialised", what);
    if (h->sh_phase != phase)
        return fail(h, PAMC_ERR_STATE, "%s out of order (expected %s next)", what,
                    h->sh_phase == 0 ? "pamc_shard_resample" : h->sh_phase == 1 ? "pamc_shard_sweep"
                                                                                : "pamc_shard_control");
    const cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    return PAMC_OK;
}

pamc_status pamc_shard_energies(pamc_handle h, int64_t *E_own) {
    pamc_status s = shard_check(h, 0, "pamc_shard_energies");
    if (s != PAMC_OK) return s;
    if (!E_own) return fail(h, PAMC_ERR_ARG, "null E_own");
    const cudaError_t e = cudaMemcpyAsync(E_own, h->d_E[h->host_t & 1], sizeof(int64_t) * (size_t)h->sh_count,
                                          cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "pamc_shard_energies");
    return PAMC_OK;
}

pamc_status pamc_shard_resample(pamc_handle h, const int64_t *E_all, int32_t *parent) {
    PAMC_RANGE("pamc_shard_resample");
    pamc_status s = shard_check(h, 0, "pamc_shard_resample");
    if (s != PAMC_OK) return s;
    if (!E_all || !parent) return fail(h, PAMC_ERR_ARG, "null E_all or parent");
    const pamc_params &p = h->p;
    const int64_t t = h->host_t;
    if (t > INT32_MAX - 2) return fail(h, PAMC_ERR_RANGE, "step counter overflow");
    if (h->dense) {   // the step's order, the population step (no cluster moves) and the tables
        pamc_params pp = p;
        pp.n_top = 0;
        cudaError_t e = launch_dense_perm(h->n, p.seed, (int32_t)t, p.sweeps, h->d_perm, h->d_pkey, h->d_sidx,
                                          h->d_boff, h->d_ctl, h->stream);
        if (e == cudaSuccess)
            e = launch_prep(pp, E_all, h->d_ctl, h->d_parent, h->d_count, h->d_ncm_idx, h->d_targets, h->d_fam,
                            nullptr, h->stream);
        if (e == cudaSuccess) e = launch_dense_tables(p.rule, h->dense_Hc, h->n, h->d_ctl, h->d_tab, h->stream);
        h->launches += 4;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(parent, h->d_parent, sizeof(int32_t) * (size_t)p.R, cudaMemcpyDeviceToHost,
                                h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "pamc_shard_resample");
        h->sh_phase = 1;
        return PAMC_OK;
    }
    if (p.sweeps > 0 && t >= h->sched_end) {
        launch_schedule(h->n, h->d_rp, h->d_adj, p.seed, (int32_t)t, kSchedSlots, p.sweeps, 0, kSchedSlots,
                        h->d_order, h->d_lvl, h->d_nlev, h->d_skey, h->d_scnt, h->stream, h->d_ell, h->ell_w,
                        h->d_pos);
        h->sched_end = t + kSchedSlots;
        h->launches += 1;
    }
    cudaError_t e = launch_prep(p, E_all, h->d_ctl, h->d_parent, h->d_count, h->d_ncm_idx, h->d_targets, h->d_fam,
                                h->d_q, h->stream, h->d_mm);
    if (e == cudaSuccess) e = launch_tables(p.kind, p.rule, h->H, h->d_ctl, h->d_tab, h->stream);
    h->launches += 3;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(parent, h->d_parent, sizeof(int32_t) * (size_t)p.R, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "pamc_shard_resample");
    h->sh_phase = 1;
    return PAMC_OK;
}

pamc_status pamc_shard_pack(pamc_handle h, const int32_t *rows, int32_t nrows, int8_t *sendbuf) {
    pamc_status s = shard_check(h, 1, "pamc_shard_pack");
    if (s != PAMC_OK) return s;
    const int32_t c = h->sh_count;
    if (nrows < 0 || nrows > h->p.R - c) return fail(h, PAMC_ERR_ARG, "nrows must be in [0, R - own slots]");
    if (nrows == 0) return PAMC_OK;
    if (!rows || !sendbuf) return fail(h, PAMC_ERR_ARG, "null rows or sendbuf");
    for (int32_t i = 0; i < nrows; ++i)
        if (rows[i] < 0 || rows[i] >= c) return fail(h, PAMC_ERR_RANGE, "row %d out of range", rows[i]);
    cudaError_t e = cudaMemcpyAsync(h->d_rows, rows, sizeof(int32_t) * (size_t)nrows, cudaMemcpyHostToDevice,
                                    h->stream);
    if (e == cudaSuccess) e = launch_gather_rows(h->n, h->d_rows, nrows, h->d_spins[h->host_t & 1], sendbuf, h->stream);
    h->launches += 1;
    if (e != cudaSuccess) return cuda_fail(h, e, "pamc_shard_pack");
    return PAMC_OK;
}

pamc_status pamc_shard_sweep(pamc_handle h, const int64_t *E_all, const int32_t *local_parent,
                             const int8_t *imports, int32_t nimports, int64_t *E_own) {
    PAMC_RANGE("pamc_shard_sweep");
    pamc_status s = shard_check(h, 1, "pamc_shard_sweep");
    if (s != PAMC_OK) return s;
    const int32_t c = h->sh_count, n = h->n;
    if (!E_all || !local_parent) return fail(h, PAMC_ERR_ARG, "null E_all or local_parent");
    if (nimports < 0 || nimports > c) return fail(h, PAMC_ERR_ARG, "nimports must be in [0, own slots]");
    if (nimports > 0 && !imports) return fail(h, PAMC_ERR_ARG, "null imports");
    for (int32_t m = 0; m < c; ++m)
        if (local_parent[m] < 0 || local_parent[m] >= c + nimports)
            return fail(h, PAMC_ERR_RANGE, "local_parent[%d] = %d out of range", m, local_parent[m]);
    const pamc_params &p = h->p;
    const int64_t t = h->host_t;
    int8_t *src = h->d_spins[t & 1], *dst = h->d_spins[(t + 1) & 1];
    int64_t *Ed = h->d_E[(t + 1) & 1];
    cudaError_t e = cudaMemcpyAsync(h->d_plocal, local_parent, sizeof(int32_t) * (size_t)c, cudaMemcpyHostToDevice,
                                    h->stream);
    if (e == cudaSuccess && nimports > 0)
        e = cudaMemcpyAsync(src + (size_t)c * n, imports, (size_t)nimports * n, cudaMemcpyDeviceToDevice, h->stream);
    if (h->dense) {   // the fields of the own slots' parents, then the sweeps
        if (e == cudaSuccess) e = dense_recompute(h, src, h->d_plocal, h->d_ncm_idx + h->sh_base, -1);
        if (e == cudaSuccess) e = sweep_timer(h, false);
        if (e == cudaSuccess)
            e = launch_dense_sweep(n, c, p.sweeps, p.rule, h->dense_Hc, (int32_t)t, p.seed, h->dense_nupd,
                                   h->dense_rows, h->dense_grid, h->d_J, h->d_perm, h->d_tab, src, h->d_plocal,
                                   nullptr, h->d_ncm_idx + h->sh_base, h->d_H, dst, Ed, h->d_G, h->d_T, h->d_T2,
                                   h->d_flip, h->d_snew, h->d_bar, h->d_ctl, h->stream, h->dense_tcu, h->sh_base);
        if (e == cudaSuccess) e = sweep_timer(h, true);
        h->launches += 4;
        if (e == cudaSuccess && E_own)
            e = cudaMemcpyAsync(E_own, Ed, sizeof(int64_t) * (size_t)c, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "pamc_shard_sweep");
        h->sh_phase = 2;
        return PAMC_OK;
    }
    if (e == cudaSuccess && p.stagnation && p.kind == 0) {
        e = launch_ncm(n, h->d_rp, h->d_adj, p, src, E_all, h->d_parent, h->d_targets, h->d_ncm_buf, h->d_nkey,
                       h->d_ctl, h->stream, h->sh_base, c, h->d_plocal);
        h->launches += 1;
    }
    pamc_params pl = p;   // the sweep sees the own slots only
    pl.R = c;
    SchedView sv{h->d_order, h->d_lvl, h->d_nlev, h->d_ell, h->d_pos, h->ell_w, h->d_nibc};
    if (e == cudaSuccess) e = sweep_timer(h, false);
    if (e == cudaSuccess)
        e = launch_sweep(sweep_kind(p), p.rule, n, h->d_rp, h->d_adj, h->H, pl, (int32_t)t,
                         (int32_t)(t % kSchedSlots), sv, h->d_tab, src, h->d_plocal, h->d_ncm_buf,
                         h->d_ncm_idx + h->sh_base, dst, Ed, h->d_ctl, h->cfg, h->W, h->stream,
                         h->gsp ? h->d_gsp : nullptr, h->sh_base, h->nib);
    if (e == cudaSuccess) e = sweep_timer(h, true);
    h->launches += 1;
    if (e == cudaSuccess && E_own)
        e = cudaMemcpyAsync(E_own, Ed, sizeof(int64_t) * (size_t)c, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "pamc_shard_sweep");
    h->sh_phase = 2;
    return PAMC_OK;
}

pamc_status pamc_shard_control(pamc_handle h, const int64_t *E_all, int64_t *E_own) {
    PAMC_RANGE("pamc_shard_control");
    pamc_status s = shard_check(h, 2, "pamc_shard_control");
    if (s != PAMC_OK) return s;
    if (!E_all) return fail(h, PAMC_ERR_ARG, "null E_all");
    const pamc_params &p = h->p;
    const int32_t c = h->sh_count, n = h->n;
    const int64_t t = h->host_t;
    int8_t *dst = h->d_spins[(t + 1) & 1];
    int64_t *Ed = h->d_E[(t + 1) & 1];
    cudaError_t e = launch_control(n, h->W, p, E_all, dst, h->d_best, h->d_ctl, h->stream, h->sh_base, c);
    h->launches += 1;
    if (e == cudaSuccess && restart_due(h)) {
        if (h->dense) {
            const int32_t tk = (int32_t)(t + 1);
            e = launch_init_spins(0, 0, n, c, p.seed, tk, 1, h->d_ctl, dst, h->stream, h->sh_base);
            if (e == cudaSuccess) e = dense_recompute(h, dst, h->d_ident, h->d_nonc, tk);
            if (e == cudaSuccess) e = launch_dense_energy(n, c, h->d_H, dst, Ed, h->d_ctl, h->stream, tk);
            h->launches += 3;
        } else {
            e = launch_init(p.kind, p.K, n, h->d_rp, h->d_adj, c, p.seed, (int32_t)(t + 1), 1, h->d_ctl, h->W, dst,
                            Ed, h->stream, h->sh_base);
            h->launches += 2;
        }
    }
    if (e == cudaSuccess && E_own)
        e = cudaMemcpyAsync(E_own, Ed, sizeof(int64_t) * (size_t)c, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "pamc_shard_control");
    h->host_t = t + 1;
    advance_z(h);
    h->sh_phase = 0;
    return PAMC_OK;
}

pamc_status pamc_shard_best(pamc_handle h, int64_t *cut, int8_t *spins, int32_t *owned) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    if (!h->initialized || !h->sharded) return fail(h, PAMC_ERR_STATE, "pamc_shard_best: no split population");
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    if (owned) *owned = c.best_owned;
    if (cut) *cut = c.mstar;
    if (spins && c.best_owned) return pamc_best(h, nullptr, spins);
    return PAMC_OK;
}

pamc_status pamc_run(pamc_handle h, const pamc_params *p) {
    pamc_status s = pamc_init(h, p);
    if (s != PAMC_OK) return s;
    s = pamc_step(h, p->steps);
    if (s != PAMC_OK) return s;
    return pamc_sync(h);
}

static pamc_status read_ctl(pamc_handle h, DevCtl &c) {
    pamc_status s = pamc_sync(h);
    if (s != PAMC_OK) return s;
    cudaError_t e = cudaMemcpy(&c, h->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "controller readback");
    return PAMC_OK;
}

pamc_status pamc_best(pamc_handle h, int64_t *cut, int8_t *spins) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_best before pamc_init");
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    if (cut) *cut = c.mstar;
    if (spins && h->sharded && !c.best_owned)
        return fail(h, PAMC_ERR_STATE, "the best configuration is held by another process (pamc_shard_best)");
    if (spins) {
        std::vector<int8_t> b(h->n);
        cudaError_t e = cudaMemcpy(b.data(), h->d_best, h->n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "best readback");
        if (h->p.kind == 0) {
            const int8_t f = b[0] < 0 ? -1 : 1;   // canonical: spin 0 is +1
            for (int32_t i = 0; i < h->n; ++i) spins[i] = (int8_t)(b[i] * f);
        } else {
            int8_t map[8] = {-1, -1, -1, -1, -1, -1, -1, -1}, next = 0;   // labels in order of first use
            for (int32_t i = 0; i < h->n; ++i) {
                const int8_t v = b[i] & 7;
                if (map[v] < 0) map[v] = next++;
                spins[i] = map[v];
            }
        }
    }
    return PAMC_OK;
}

pamc_status pamc_state(pamc_handle h, int8_t *spins, int64_t *E, int32_t *parents, int32_t *counts) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_state before pamc_init");
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    if (h->sharded && h->sh_phase != 0)
        return fail(h, PAMC_ERR_STATE, "pamc_state in the middle of a split-population step");
    const int cur = c.t & 1;
    // a split population: the own slots (their parents as indices into all R)
    const size_t R = (size_t)(h->sharded ? h->sh_count : h->p.R);
    const size_t off = h->sharded ? (size_t)h->sh_base : 0;
    cudaError_t e = cudaSuccess;
    if (spins) e = cudaMemcpy(spins, h->d_spins[cur], R * h->n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && E) e = cudaMemcpy(E, h->d_E[cur], R * sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && parents)
        e = cudaMemcpy(parents, h->d_parent + off, R * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && counts)
        e = cudaMemcpy(counts, h->d_count + off, R * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "state readback");
    return PAMC_OK;
}

// ---------------------------------------------------------------- checkpoints
namespace {

// The whole state of Algorithm 1 at the start of iteration t: the
// parameters, the controller (beta, Delta, z, cycle, cooldown, flags, M*
// history, M*, counters), the population and its energies, the last
// iteration's parents and copy counts, the lineage and the best
// configuration.  Every random draw is keyed by (seed, t, ...), so a run
// continued from it is the uninterrupted run.
struct CkptHeader {
    char magic[8];
    uint32_t version, ctl_bytes;
    int32_t dense, n, nnz, H;
    int64_t W;
    uint64_t inst_hash;
    pamc_params p;
};
constexpr uint32_t kCkptVersion = 1;

size_t ckpt_bytes(int32_t n, int32_t R) {
    return sizeof(CkptHeader) + sizeof(DevCtl) + (size_t)R * n + (size_t)R * 8 + (size_t)R * 4 * 4 + (size_t)n;
}

}  // namespace

pamc_status pamc_save(pamc_handle h, void *buf, size_t capacity, size_t *size) {
    PAMC_RANGE("pamc_save");
    if (!h || !size) return fail(h, PAMC_ERR_ARG, "null handle or size");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_save before pamc_init");
    if (h->sharded) return fail(h, PAMC_ERR_STATE, "pamc_save: the population is split over processes");
    const int32_t n = h->n, R = h->p.R;
    *size = ckpt_bytes(n, R);
    if (!buf) return PAMC_OK;
    if (capacity < *size) return fail(h, PAMC_ERR_RANGE, "checkpoint needs %zu bytes", *size);
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    const int cur = c.t & 1;
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "PAMCCKPT", 8);
    hd.version = kCkptVersion;
    hd.ctl_bytes = (uint32_t)sizeof(DevCtl);
    hd.dense = h->dense;
    hd.n = n; hd.nnz = h->nnz; hd.H = h->H; hd.W = h->W;
    hd.inst_hash = h->inst_hash;
    hd.p = h->p;
    char *o = static_cast<char *>(buf);
    memcpy(o, &hd, sizeof(hd));
    o += sizeof(hd);
    memcpy(o, &c, sizeof(c));
    o += sizeof(c);
    cudaError_t e = cudaMemcpy(o, h->d_spins[cur], (size_t)R * n, cudaMemcpyDeviceToHost);
    o += (size_t)R * n;
    if (e == cudaSuccess) e = cudaMemcpy(o, h->d_E[cur], (size_t)R * 8, cudaMemcpyDeviceToHost);
    o += (size_t)R * 8;
    if (e == cudaSuccess) e = cudaMemcpy(o, h->d_parent, (size_t)R * 4, cudaMemcpyDeviceToHost);
    o += (size_t)R * 4;
    if (e == cudaSuccess) e = cudaMemcpy(o, h->d_count, (size_t)R * 4, cudaMemcpyDeviceToHost);
    o += (size_t)R * 4;
    if (e == cudaSuccess) e = cudaMemcpy(o, h->d_fam, (size_t)R * 8, cudaMemcpyDeviceToHost);
    o += (size_t)R * 8;
    if (e == cudaSuccess) e = cudaMemcpy(o, h->d_best, (size_t)n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "pamc_save readback");
    return PAMC_OK;
}

pamc_status pamc_load(pamc_handle h, const void *buf, size_t size) {
    PAMC_RANGE("pamc_load");
    if (!h || !buf) return fail(h, PAMC_ERR_ARG, "null handle or buffer");
    if (size < sizeof(CkptHeader)) return fail(h, PAMC_ERR_ARG, "not a checkpoint (too short)");
    CkptHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    if (memcmp(hd.magic, "PAMCCKPT", 8) != 0 || hd.version != kCkptVersion || hd.ctl_bytes != sizeof(DevCtl))
        return fail(h, PAMC_ERR_ARG, "not a checkpoint of this library version");
    if (hd.dense != h->dense || hd.n != h->n || hd.nnz != h->nnz || hd.H != h->H || hd.W != h->W ||
        hd.inst_hash != h->inst_hash)
        return fail(h, PAMC_ERR_ARG, "the checkpoint belongs to another instance");
    const int32_t n = h->n, R = hd.p.R;
    if (R < 1 || R > kMaxPopulation || size != ckpt_bytes(n, R))
        return fail(h, PAMC_ERR_ARG, "checkpoint size mismatch");
    DevCtl c;
    const char *in = static_cast<const char *>(buf) + sizeof(hd);
    memcpy(&c, in, sizeof(c));
    in += sizeof(c);
    if (c.t < 0 || c.t > INT32_MAX - 2) return fail(h, PAMC_ERR_RANGE, "checkpoint step index out of range");
    const int8_t *spins = reinterpret_cast<const int8_t *>(in);
    for (size_t x = 0; x < (size_t)R * n; ++x) {
        const int8_t v = spins[x];
        const bool ok = hd.p.kind == 0 ? (v == 1 || v == -1) : (v >= 0 && v < (hd.p.K ? hd.p.K : 3));
        if (!ok) return fail(h, PAMC_ERR_RANGE, "checkpoint spin %zu out of range", x);
    }
    const int32_t *ints = reinterpret_cast<const int32_t *>(in + (size_t)R * n + (size_t)R * 8);
    for (size_t x = 0; x < (size_t)R * 4; ++x)      // parents, counts, two lineage rows
        if (ints[x] < 0 || ints[x] > R) return fail(h, PAMC_ERR_RANGE, "checkpoint index out of range");
    pamc_status s = init_run(h, &hd.p, 0, 0);
    if (s != PAMC_OK) return s;
    const int cur = c.t & 1;
    cudaError_t e = cudaMemcpyAsync(h->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_spins[cur], in, (size_t)R * n, cudaMemcpyHostToDevice, h->stream);
    in += (size_t)R * n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_E[cur], in, (size_t)R * 8, cudaMemcpyHostToDevice, h->stream);
    in += (size_t)R * 8;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_parent, in, (size_t)R * 4, cudaMemcpyHostToDevice, h->stream);
    in += (size_t)R * 4;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_count, in, (size_t)R * 4, cudaMemcpyHostToDevice, h->stream);
    in += (size_t)R * 4;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_fam, in, (size_t)R * 8, cudaMemcpyHostToDevice, h->stream);
    in += (size_t)R * 8;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_best, in, (size_t)n, cudaMemcpyHostToDevice, h->stream);
    // dense runs keep the fields of the population: recompute them exactly
    if (e == cudaSuccess && h->dense) e = dense_recompute(h, h->d_spins[cur], h->d_ident, h->d_nonc, -1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // the host buffer may go after return
    if (e != cudaSuccess) return cuda_fail(h, e, "pamc_load upload");
    h->host_t = c.t;
    h->host_z = c.z;
    h->sched_end = c.t;   // the next step builds the schedules from step t on
    h->launches += h->dense ? 1 : 0;
    return PAMC_OK;
}

pamc_status pamc_set_population(pamc_handle h, const int8_t *spins) {
    if (!h || !spins) return fail(h, PAMC_ERR_ARG, "null argument");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_set_population before pamc_init");
    if (h->sharded) return fail(h, PAMC_ERR_STATE, "pamc_set_population: the population is split over processes");
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    if (c.done) return fail(h, PAMC_ERR_STATE, "the run has reached its target");
    const int32_t n = h->n, R = h->p.R;
    const size_t total = (size_t)R * n;
    for (size_t x = 0; x < total; ++x) {
        const int8_t v = spins[x];
        const bool ok = h->p.kind == 0 ? (v == 1 || v == -1) : (v >= 0 && v < h->p.K);
        if (!ok) return fail(h, PAMC_ERR_RANGE, "spin %zu out of range", x);
    }
    const int cur = c.t & 1;
    cudaError_t e = cudaMemcpyAsync(h->d_spins[cur], spins, total, cudaMemcpyHostToDevice, h->stream);
    if (h->dense) {
        if (e == cudaSuccess)
            e = dense_recompute(h, h->d_spins[cur], h->d_ident, h->d_nonc, -1);
        if (e == cudaSuccess)
            e = launch_dense_energy(n, R, h->d_H, h->d_spins[cur], h->d_E[cur], h->d_ctl, h->stream, -1);
    } else if (e == cudaSuccess) {
        e = launch_energy(h->p.kind, n, h->d_rp, h->d_adj, R, h->d_ctl, h->W, h->d_spins[cur], h->d_E[cur],
                          h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set population");
    h->launches += 2;
    return PAMC_OK;
}

pamc_status pamc_dense_rows(pamc_handle h, int64_t *rows_gathered, int64_t *positions_visited) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    if (!h->dense) return fail(h, PAMC_ERR_ARG, "pamc_dense_rows: not a dense instance");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_dense_rows before pamc_init");
    cudaError_t e = cudaSetDevice(h->device);
    DevCtl c;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c, h->d_ctl, sizeof(c), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "pamc_dense_rows");
    if (rows_gathered) *rows_gathered = c.dense_rows;
    if (positions_visited) *positions_visited = c.dense_positions;
    return PAMC_OK;
}

pamc_status pamc_fields(pamc_handle h, int32_t *H) {
    if (!h || !H) return fail(h, PAMC_ERR_ARG, "null argument");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_fields before pamc_init");
    if (!h->dense) return fail(h, PAMC_ERR_ARG, "sparse runs keep no field array (fields are pulled per visit)");
    pamc_status s = pamc_sync(h);
    if (s != PAMC_OK) return s;
    const cudaError_t e = cudaMemcpy(H, h->d_H, sizeof(int32_t) * (size_t)h->p.R * h->n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "fields readback");
    return PAMC_OK;
}

pamc_status pamc_control_state(pamc_handle h, int64_t *iv, double *dv) {
    if (!h || !iv || !dv) return fail(h, PAMC_ERR_ARG, "null argument");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_control_state before pamc_init");
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    iv[0] = c.t; iv[1] = c.z; iv[2] = c.cycle; iv[3] = c.cooldown; iv[4] = c.enable_cm;
    iv[5] = c.done; iv[6] = c.ncm_last; iv[7] = c.hist_len; iv[8] = c.ncm_flipped;
    iv[9] = c.ncm_dE_max;
    dv[0] = c.beta; dv[1] = c.delta;
    return PAMC_OK;
}

pamc_status pamc_control_history(pamc_handle h, int64_t *hist, int32_t *hist_len, int64_t *mstar) {
    if (!h || !hist_len) return fail(h, PAMC_ERR_ARG, "null argument");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_control_history before pamc_init");
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    *hist_len = c.hist_len;
    if (hist)
        for (int32_t i = 0; i < c.hist_len && i < kHistMax; ++i) hist[i] = c.hist[i];
    if (mstar) *mstar = c.mstar;
    return PAMC_OK;
}

pamc_status pamc_hamming(pamc_handle h, int64_t *hist, int64_t *sum) {
    if (!h || !hist || !sum) return fail(h, PAMC_ERR_ARG, "null argument");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_hamming before pamc_init");
    if (h->sharded) return fail(h, PAMC_ERR_STATE, "pamc_hamming: the population is split over processes");
    if (h->p.kind != 0) return fail(h, PAMC_ERR_ARG, "Hamming distances are defined for Ising (Max-Cut) runs");
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    const int32_t n = h->n, R = h->p.R;
    const size_t nb = (size_t)n / 2 + 1, nw = ((size_t)n + 31) / 32;
    std::vector<DevBuf> tmp;
    uint32_t *bits = nullptr;
    uint8_t *sb = nullptr;
    unsigned long long *dh = nullptr;
    const bool tc = hamming_tc_enabled(n, R);   // overlaps on the tensor cores, else XOR-popcount
    const bool ok = tc ? alloc_n(h, sb, hamming_tc_scratch(n, R), tmp)
                       : alloc_n(h, bits, std::max<size_t>((size_t)R * nw, 1), tmp);
    if (!ok || !alloc_n(h, dh, nb + 1, tmp)) {
        dev_free_all(h, tmp);
        return fail(h, PAMC_ERR_OOM, "device allocation for the Hamming distances failed");
    }
    int *err = reinterpret_cast<int *>(reinterpret_cast<char *>(h->d_ctl) + offsetof(DevCtl, err));
    cudaError_t e = tc ? launch_hamming_tc(n, R, h->d_spins[c.t & 1], sb, dh, dh + nb, err, h->stream)
                       : launch_hamming(n, R, h->d_spins[c.t & 1], bits, dh, dh + nb, h->stream);
    std::vector<unsigned long long> out(nb + 1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.data(), dh, sizeof(unsigned long long) * (nb + 1), cudaMemcpyDeviceToHost,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free_all(h, tmp);
    if (e != cudaSuccess) return cuda_fail(h, e, "Hamming distances");
    s = pamc_sync(h);   // a bounded wait of the tensor-core kernel that gave up is reported here
    if (s != PAMC_OK) return s;
    for (size_t k = 0; k < nb; ++k) hist[k] = (int64_t)out[k];
    *sum = (int64_t)out[nb];
    return PAMC_OK;
}

pamc_status pamc_lineage(pamc_handle h, int32_t *family, int32_t *n_families) {
    if (!h || !family) return fail(h, PAMC_ERR_ARG, "null argument");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_lineage before pamc_init");
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    const int32_t R = h->p.R;
    cudaError_t e = cudaMemcpy(family, h->d_fam + (size_t)(c.t & 1) * R, sizeof(int32_t) * R,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "lineage readback");
    if (n_families) {
        std::vector<char> seen(R, 0);
        int32_t k = 0;
        for (int32_t r = 0; r < R; ++r)
            if (family[r] >= 0 && family[r] < R && !seen[family[r]]) { seen[family[r]] = 1; ++k; }
        *n_families = k;
    }
    return PAMC_OK;
}

int64_t pamc_launch_count(pamc_handle h) { return h ? h->launches : 0; }

pamc_status pamc_sweep_shape(pamc_handle h, int *groups_per_cta, int *warps_per_group, int *lanes_per_vertex) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    if (!h->initialized || h->dense) return fail(h, PAMC_ERR_STATE, "no sparse run initialised");
    if (groups_per_cta) *groups_per_cta = h->cfg.groups_per_cta;
    if (warps_per_group) *warps_per_group = h->cfg.warps_per_group;
    if (lanes_per_vertex) *lanes_per_vertex = h->cfg.lanes_per_vertex;
    return PAMC_OK;
}

pamc_status pamc_set_sweep_timing(pamc_handle h, int on) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    h->time_sweeps = on != 0;
    return PAMC_OK;
}

pamc_status pamc_sweep_stats(pamc_handle h, int64_t *flips, int64_t *launches, double *ms) {
    if (!h) return fail(h, PAMC_ERR_ARG, "null handle");
    if (!h->initialized) return fail(h, PAMC_ERR_STATE, "pamc_sweep_stats before pamc_init");
    DevCtl c;
    pamc_status s = read_ctl(h, c);
    if (s != PAMC_OK) return s;
    const cudaError_t e = fold_sweep_events(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "sweep timing");
    if (flips) *flips = c.sweep_flips;
    if (launches) *launches = h->sweep_timed;
    if (ms) *ms = h->sweep_ms;
    h->sweep_timed = 0;
    h->sweep_ms = 0.0;
    return PAMC_OK;
}

pamc_status pamc_sweep_mode(pamc_handle h, int *mode) {
    if (!h || !mode) return fail(h, PAMC_ERR_ARG, "null argument");
    if (!h->initialized || h->dense || h->p.kind != 0)
        return fail(h, PAMC_ERR_STATE, "no sparse Ising run initialised");
    const bool ell = h->d_ell != nullptr;
    if (h->gsp) *mode = (ell ? 1 : 0) | 4;
    else if (h->nib) *mode = 1 | 16;
    else *mode = sweep_push_ok(h->H, h->p.sweeps, ell, h->cfg.lanes_per_vertex) ? 2 : ell ? 1 : 0;
    if (h->H > kByteLaneMaxH) *mode |= 8;
    return PAMC_OK;
}

int64_t pamc_weight_sum(pamc_handle h) { return h ? h->W : 0; }

pamc_status pamc_last_error(pamc_handle h, char *buf, size_t len) {
    if (!buf || len == 0) return PAMC_ERR_ARG;
    snprintf(buf, len, "%s", h ? h->err : g_create_err);
    return PAMC_OK;
}

void pamc_destroy(pamc_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    release_run(h);
    for (cudaEvent_t ev : h->sweep_ev) cudaEventDestroy(ev);
    dev_free_all(h, h->inst_bufs);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------- batches
// A batch advances many sparse Ising instances together.  Every launch reads
// the member's step index from its device controller (ctl->t), so the
// launches of one step are the same for every step: they are captured once
// per membership into a CUDA graph and replayed.  Members that reached their
// last step are no-ops inside the graph until the next rebuild drops them.
struct pamc_batch_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<pamc_handle> members;
    bool dirty = true;
    DevBuf sw, swi, sd, sdi, prep, tabs, ctl;
    DevBuf ncm, ncmi, rd, rdi;   // cluster moves and restart re-draws of the members that have them
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t graph_launches = 0;   // kernel launches in one replay
    int64_t launches = 0;
    int64_t rebuilds = 0;
    SweepCfg shape[3];            // batched sweep launch shape per size class
    bool global[3] = {false, false, false};   // Ising members' spin words in device memory
    char err[256] = "";
};

namespace {

pamc_status bfail(pamc_batch b, pamc_status s, const char *fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) snprintf(b->err, sizeof(b->err), "%s", buf);
    else snprintf(g_create_err, sizeof(g_create_err), "%s", buf);
    return s;
}

// Stream-ordered upload of a descriptor array (the stream's earlier work,
// which may still read the old contents, completes first).
template <typename T>
bool upload(pamc_batch b, DevBuf &buf, const std::vector<T> &v) {
    const size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
    if (buf.bytes < bytes) {
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return false;
        if (buf.p) cudaFree(buf.p);
        buf.p = nullptr;
        buf.bytes = 0;
        if (cudaMalloc(&buf.p, bytes * 2) != cudaSuccess) { cudaGetLastError(); return false; }
        buf.bytes = bytes * 2;
    }
    if (v.empty()) return true;
    if (cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return false;
    // the host vector is reused by the next rebuild
    return cudaStreamSynchronize(b->stream) == cudaSuccess;
}

// Sweep launch shape per size class of n (groups of 4 replicas per CTA,
// warps per group).  Small instances pack several groups into one CTA.
constexpr int kClasses = 3;
int batch_class(int32_t n) { return n <= 2048 ? 0 : n <= 8192 ? 1 : 2; }
bool batch_lanes_ok(int l) { return l == 1 || l == 2 || l == 4; }
SweepCfg batch_cfg(int cls) {
    static const SweepCfg c[kClasses] = {{8, 1, 1}, {4, 2, 1}, {1, 16, 1}};
    const char *env = getenv("PAMC_BATCH_CFG");   // "g0,w0;g1,w1;g2,w2"
    if (env) {
        int v[6];
        if (sscanf(env, "%d,%d;%d,%d;%d,%d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 6) {
            SweepCfg o{v[2 * cls], v[2 * cls + 1], 1};
            if (o.groups_per_cta >= 1 && o.warps_per_group >= 1 && o.groups_per_cta * o.warps_per_group <= 32)
                return o;
        }
    }
    return c[cls];
}

void drop_graph(pamc_batch b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Descriptor arrays for the members that still have steps left, then the
// captured launch sequence of one step.
pamc_status rebuild(pamc_batch b) {
    drop_graph(b);
    std::vector<SchedDesc> sd;
    std::vector<int2> sdi;
    std::vector<PrepDesc> prep;
    std::vector<TabDesc> tabs;
    std::vector<CtlDesc> ctls;
    std::vector<SweepDesc> sw;
    std::vector<int2> swi[2][2][kClasses];   // Ising, spin words on chip [ell][rule][class]
    std::vector<int2> gswi[2][2][kClasses];  // Ising, spin words in device memory
    std::vector<int2> pswi[2][kClasses];     // Potts (cascaded sampler) [ell][class]
    std::vector<int2> nswi[2][2][kClasses];  // Ising, 4-bit lanes (ELL rows) [biased][rule][class]
    std::vector<NcmDesc> ncm;
    std::vector<int2> ncmi;
    std::vector<RedrawDesc> rds;
    std::vector<int2> rdsi, rdei;             // re-draw items: (member, chunk of draws), (member, replica)
    int32_t ncm_nmax = 1;
    int32_t nmax[kClasses] = {0, 0, 0}, pnmax[kClasses] = {0, 0, 0}, gnmax[kClasses] = {0, 0, 0},
            nnmax[kClasses] = {0, 0, 0}, Rmax = 1;
    auto member_global = [&](pamc_handle h) { return h->p.kind == 0 && (h->gsp || b->global[batch_class(h->n)]); };
    // members whose field ranges fit 4-bit lanes take eight replicas a word, as alone
    auto member_nib = [&](pamc_handle h) {
        return h->p.kind == 0 && !member_global(h) &&
               sweep_nibble_ok(h->H, h->p.sweeps, h->ell_w, 1, false, h->d_nibc != nullptr) && !sweep_push_enabled();
    };
    for (pamc_handle h : b->members)
        if (h->host_t < h->p.steps) {
            int32_t &m = (h->p.kind != 0 ? pnmax : member_global(h) ? gnmax : member_nib(h) ? nnmax
                                                                                            : nmax)[batch_class(h->n)];
            m = std::max(m, h->n);
        }
    // the shape of each class, with fewer groups per CTA where the largest
    // member's spins (Ising: 4n bytes a group, Potts: 8n) need it
    SweepCfg eff[kClasses], peff[kClasses], geff[kClasses], neff[kClasses];
    for (int c = 0; c < kClasses; ++c) {
        neff[c] = SweepCfg{b->shape[c].groups_per_cta, b->shape[c].warps_per_group, 1};
        while (neff[c].groups_per_cta > 1 && sweep_nibble_smem_bytes(nnmax[c], kNibbleBiasedMaxH, neff[c]) > kSmemMax)
            neff[c].groups_per_cta -= 1;
        geff[c] = SweepCfg{b->shape[c].groups_per_cta, b->shape[c].warps_per_group, 1};
        eff[c] = b->shape[c];
        while (eff[c].groups_per_cta > 1 && sweep_ising_smem_bytes(nmax[c], 127, eff[c]) > kSmemMax)
            eff[c].groups_per_cta -= 1;
        peff[c] = SweepCfg{b->shape[c].groups_per_cta, b->shape[c].warps_per_group, 1};
        while (peff[c].groups_per_cta > 1 && sweep_potts_smem_bytes(pnmax[c], 127, peff[c]) > kSmemMax)
            peff[c].groups_per_cta -= 1;
    }
    for (pamc_handle h : b->members) {
        const pamc_params &p = h->p;
        if (h->host_t >= p.steps) continue;
        const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
        const int32_t t_end = p.steps;
        if (p.sweeps > 0) {
            SchedDesc d{h->d_rp, h->d_adj, h->d_order, h->d_lvl, h->d_nlev, h->d_scnt, h->d_skey, h->d_ell,
                        h->d_pos, h->n, 0, p.sweeps, kSchedSlots, h->ell_w, k0, k1, h->d_ctl,
                        kSchedSlots - 1, t_end};
            const int idx = (int)sd.size();
            sd.push_back(d);
            for (int x = 0; x < p.sweeps; ++x) sdi.push_back(make_int2(idx, x));
        }
        PrepDesc pd{nullptr, h->d_ctl, h->d_parent, h->d_count, h->d_ncm_idx, h->d_targets, p.R,
                    p.kind, p.resample, p.n_top, p.cooldown_tau, k0, k1, {h->d_E[0], h->d_E[1]}, t_end,
                    h->d_fam, p.z_rst > 0 && p.restart_reinit ? 1 : 0};
        prep.push_back(pd);
        if (p.stagnation && p.kind == 0) {   // the cluster moves of the member's targets
            NcmDesc nd{h->d_rp, h->d_adj, h->d_parent, h->d_targets, h->d_ncm_buf, h->d_nkey, h->d_ctl,
                       {h->d_spins[0], h->d_spins[1]}, {h->d_E[0], h->d_E[1]}, h->n, p.R, p.n_top,
                       p.mis_trials, t_end, k0, k1};
            const int nidx = (int)ncm.size();
            ncm.push_back(nd);
            for (int32_t q = 0; q < std::min(p.n_top, p.R); ++q) ncmi.push_back(make_int2(nidx, q));
            ncm_nmax = std::max(ncm_nmax, h->n);
        }
        if (p.z_rst > 0 && p.restart_reinit) {   // a restart's re-draw
            RedrawDesc rdd{h->d_rp, h->d_adj, h->d_ctl, {h->d_spins[0], h->d_spins[1]}, {h->d_E[0], h->d_E[1]},
                           h->W, h->n, p.R, p.kind, p.K, k0, k1};
            const int ridx = (int)rds.size();
            rds.push_back(rdd);
            const size_t total = (size_t)((p.R + 3) / 4) * h->n, chunk = (size_t)256 * kRedrawPerThread;
            for (size_t c = 0; c * chunk < total; ++c) rdsi.push_back(make_int2(ridx, (int)c));
            for (int32_t r = 0; r < p.R; ++r) rdei.push_back(make_int2(ridx, r));
        }
        tabs.push_back(TabDesc{h->d_ctl, h->d_tab, p.rule, h->H, t_end, p.kind});
        SweepDesc d;
        memset(&d, 0, sizeof(d));
        d.rp = h->d_rp; d.adj = h->d_adj; d.sorder = h->d_order; d.slvl = h->d_lvl; d.snlev = h->d_nlev;
        d.sell = h->d_ell; d.spos = h->d_pos; d.tab = h->d_tab; d.parent = h->d_parent;
        d.ncm_buf = h->d_ncm_buf; d.ncm_idx = h->d_ncm_idx; d.ctl = h->d_ctl;
        d.n = h->n; d.n_pad = (h->n + 3) & ~3; d.H = h->H; d.R = p.R; d.S = p.sweeps;
        d.W = h->ell_w; d.K = make_philox_keys(p.seed);
        d.sp[0] = h->d_spins[0]; d.sp[1] = h->d_spins[1]; d.en[0] = h->d_E[0]; d.en[1] = h->d_E[1];
        d.slots = kSchedSlots; d.t_end = t_end; d.Wsum = h->W;
        const int cls = batch_class(h->n);
        const bool gl = member_global(h);
        if (gl && !h->d_gsp && !alloc_n(h, h->d_gsp, gsp_words(h->n, p.R), h->bufs))
            return bfail(b, PAMC_ERR_OOM, "device allocation of a member's group spin words failed");
        d.gsp = gl ? h->d_gsp : nullptr;
        const bool nb = member_nib(h);
        d.nibc = nb ? h->d_nibc : nullptr;
        const SweepCfg cfg = p.kind != 0 ? peff[cls] : gl ? geff[cls] : nb ? neff[cls] : eff[cls];
        d.push = p.kind == 0 && !gl && !nb && sweep_push_ok(h->H, p.sweeps, h->d_ell != nullptr, cfg.lanes_per_vertex)
                     ? 1 : 0;
        const int idx = (int)sw.size();
        sw.push_back(d);
        const int32_t groups = nb ? (p.R + 7) / 8 : (p.R + 3) / 4;
        const int32_t ctas = (groups + cfg.groups_per_cta - 1) / cfg.groups_per_cta;
        // with sweeps = 0 the launch still copies the resampled population and its energies
        auto &items = p.kind != 0 ? pswi[h->d_ell != nullptr][cls]
                                  : nb ? nswi[h->d_nibc != nullptr][p.rule][cls]
                                       : (gl ? gswi : swi)[h->d_ell != nullptr][p.rule][cls];
        for (int32_t x = 0; x < ctas; ++x) items.push_back(make_int2(idx, x));
        Rmax = std::max(Rmax, p.R);
        CtlDesc c{nullptr, nullptr, h->d_best, h->d_ctl, h->W, p.target_cut, p.reheat_factor, p.beta0,
                  h->n, p.R, p.stagnation, p.z_rst, p.win_short, p.win_long, p.max_distinct_short,
                  p.max_distinct_long, {h->d_E[0], h->d_E[1]}, {h->d_spins[0], h->d_spins[1]}, t_end};
        ctls.push_back(c);
    }
    std::vector<int2> all_items;
    for (auto &a : swi)
        for (auto &c : a)
            for (auto &v : c) all_items.insert(all_items.end(), v.begin(), v.end());
    for (auto &a : gswi)
        for (auto &c : a)
            for (auto &v : c) all_items.insert(all_items.end(), v.begin(), v.end());
    for (auto &a : pswi)
        for (auto &v : a) all_items.insert(all_items.end(), v.begin(), v.end());
    for (auto &a : nswi)
        for (auto &c : a)
            for (auto &v : c) all_items.insert(all_items.end(), v.begin(), v.end());
    const size_t n_rdsi = rdsi.size();
    rdsi.insert(rdsi.end(), rdei.begin(), rdei.end());   // one upload: spin items, then energy items
    const bool ok = upload(b, b->sd, sd) && upload(b, b->sdi, sdi) && upload(b, b->prep, prep) &&
                    upload(b, b->tabs, tabs) && upload(b, b->sw, sw) && upload(b, b->ctl, ctls) &&
                    upload(b, b->swi, all_items) && upload(b, b->ncm, ncm) && upload(b, b->ncmi, ncmi) &&
                    upload(b, b->rd, rds) && upload(b, b->rdi, rdsi);
    if (!ok) return bfail(b, PAMC_ERR_CUDA, "descriptor upload failed");
    b->dirty = false;
    b->graph_launches = 0;
    if (prep.empty()) return PAMC_OK;
    // one step: population step + tables, sweeps per (ELL, rule, class), controller, next schedule
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return bfail(b, PAMC_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    int32_t nl = 0;
    e = launch_population_batched((const PrepDesc *)b->prep.p, (const TabDesc *)b->tabs.p, (int32_t)prep.size(),
                                  Rmax, b->stream);
    nl += 2;
    if (e == cudaSuccess && !ncmi.empty()) {
        e = launch_ncm_batched((const NcmDesc *)b->ncm.p, (const int2 *)b->ncmi.p, (int32_t)ncmi.size(), ncm_nmax,
                               b->stream);
        nl += 1;
    }
    size_t off = 0;
    for (int el = 0; el < 2 && e == cudaSuccess; ++el)
        for (int ru = 0; ru < 2 && e == cudaSuccess; ++ru)
            for (int c = 0; c < kClasses && e == cudaSuccess; ++c) {
                const auto &items = swi[el][ru][c];
                if (items.empty()) continue;
                e = launch_sweep_ising_batched(ru, el != 0, (const SweepDesc *)b->sw.p, (const int2 *)b->swi.p + off,
                                               (int32_t)items.size(), nmax[c], eff[c], b->stream);
                off += items.size();
                nl += 1;
            }
    for (int el = 0; el < 2 && e == cudaSuccess; ++el)
        for (int ru = 0; ru < 2 && e == cudaSuccess; ++ru)
            for (int c = 0; c < kClasses && e == cudaSuccess; ++c) {
                const auto &items = gswi[el][ru][c];
                if (items.empty()) continue;
                e = launch_sweep_ising_batched(ru, el != 0, (const SweepDesc *)b->sw.p, (const int2 *)b->swi.p + off,
                                               (int32_t)items.size(), gnmax[c], geff[c], b->stream, true);
                off += items.size();
                nl += 1;
            }
    for (int el = 0; el < 2 && e == cudaSuccess; ++el)
        for (int c = 0; c < kClasses && e == cudaSuccess; ++c) {
            const auto &items = pswi[el][c];
            if (items.empty()) continue;
            e = launch_sweep_potts_batched(el != 0, (const SweepDesc *)b->sw.p, (const int2 *)b->swi.p + off,
                                           (int32_t)items.size(), pnmax[c], peff[c], b->stream);
            off += items.size();
            nl += 1;
        }
    for (int bi = 0; bi < 2 && e == cudaSuccess; ++bi)
        for (int ru = 0; ru < 2 && e == cudaSuccess; ++ru)
            for (int c = 0; c < kClasses && e == cudaSuccess; ++c) {
                const auto &items = nswi[bi][ru][c];
                if (items.empty()) continue;
                e = launch_sweep_ising_nib_batched(ru, bi != 0, (const SweepDesc *)b->sw.p,
                                                   (const int2 *)b->swi.p + off, (int32_t)items.size(), nnmax[c],
                                                   neff[c], b->stream);
                off += items.size();
                nl += 1;
            }
    if (e == cudaSuccess) e = launch_control_batched((const CtlDesc *)b->ctl.p, (int32_t)ctls.size(), b->stream);
    nl += 1;
    if (e == cudaSuccess && !rds.empty()) {
        e = launch_redraw_batched((const RedrawDesc *)b->rd.p, (int32_t)rds.size(), (const int2 *)b->rdi.p,
                                  (int32_t)n_rdsi, (const int2 *)b->rdi.p + n_rdsi, (int32_t)rdei.size(), b->stream);
        nl += 3;
    }
    if (e == cudaSuccess && !sdi.empty()) {
        int32_t sched_nmax = 1;
        for (const SchedDesc &d : sd) sched_nmax = std::max(sched_nmax, d.n);
        launch_schedule_batched((const SchedDesc *)b->sd.p, (const int2 *)b->sdi.p, (int32_t)sdi.size(), sched_nmax,
                                b->stream);
        e = cudaGetLastError();
        nl += 1;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, PAMC_ERR_CUDA, "capture of the batch step: %s", cudaGetErrorString(e));
    }
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        drop_graph(b);
        return bfail(b, PAMC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    b->graph_launches = nl;
    b->rebuilds += 1;
    return PAMC_OK;
}

}  // namespace

extern "C" {

size_t pamc_footprint(pamc_handle h, const pamc_params *p) {
    if (!h || !p || h->dense) return 0;
    const size_t n = (size_t)h->n, R = (size_t)std::max(p->R, 1), S = (size_t)std::max(p->sweeps, 1);
    const size_t slots = kSchedSlots;
    size_t b = 2 * R * n + 3 * R * 8 + 4 * R * 4 + 2 * R * 4 + n;
    b += slots * S * (n * 4 + (n + 1) * 4 + 4 + n * 4 + n * 4);
    if (h->ell_w > 0) b += slots * S * (((n + 31) / 32) * 32 * (size_t)h->ell_w * 4 + n * 8);
    b += (size_t)(p->kind == 0 ? 2 * h->H + 1 : (4 * h->H + 1) * (4 * h->H + 1) + 4 * h->H + 1) * 8;
    if (p->stagnation && p->kind == 0) b += 5 * (size_t)std::min(p->n_top > 0 ? p->n_top : std::max(1, p->R / 16), p->R) * n;
    b += ((size_t)h->n + 1) * 4 + (size_t)std::max(h->nnz, 1) * 4;   // the instance itself
    // Ising groups whose spin words do not fit shared memory keep them in device memory
    if (p->kind == 0 && sweep_smem_bytes(0, (int32_t)n, h->H, SweepCfg{1, 1, 1}) > kSmemMax)
        b += gsp_words((int32_t)n, p->R) * 4 * (h->H > kByteLaneMaxH ? 2 : 1);
    return b + sizeof(DevCtl);
}

pamc_status pamc_batch_create(int cuda_device, void *stream, pamc_batch *out) {
    if (!out) return bfail(nullptr, PAMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (cudaSetDevice(cuda_device) != cudaSuccess) return bfail(nullptr, PAMC_ERR_CUDA, "cudaSetDevice failed");
    pamc_batch b = new (std::nothrow) pamc_batch_s();
    if (!b) return bfail(nullptr, PAMC_ERR_OOM, "host allocation failed");
    b->device = cuda_device;
    b->stream = (cudaStream_t)stream;
    for (int c = 0; c < kClasses; ++c) b->shape[c] = batch_cfg(c);
    if (!b->stream) {   // graph capture needs a stream other than the legacy default one
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return bfail(nullptr, PAMC_ERR_CUDA, "stream creation failed");
        }
        b->own_stream = true;
    }
    *out = b;
    return PAMC_OK;
}

pamc_status pamc_batch_add(pamc_batch b, pamc_handle h) {
    if (!b || !h) return bfail(b, PAMC_ERR_ARG, "null batch or handle");
    if (!h->initialized) return bfail(b, PAMC_ERR_STATE, "handle not initialised (pamc_init)");
    if (h->dense) return bfail(b, PAMC_ERR_ARG, "batches hold sparse instances");
    if (h->sharded) return bfail(b, PAMC_ERR_ARG, "a split population cannot join a batch");
    if (h->p.R > kPrepOneCtaMaxR)
        return bfail(b, PAMC_ERR_ARG, "batched members have at most %d replicas", kPrepOneCtaMaxR);
    if (h->H > kByteLaneMaxH)
        return bfail(b, PAMC_ERR_ARG, "batched members need sum_j |w_ij| <= %d", kByteLaneMaxH);
    if (h->p.kind == 1 && h->p.rule != 0)
        return bfail(b, PAMC_ERR_ARG, "batched Max-3-Cut members use the cascaded sampler (rule 0)");
    if (h->device != b->device) return bfail(b, PAMC_ERR_ARG, "handle on another device");
    for (pamc_handle m : b->members)
        if (m == h) return bfail(b, PAMC_ERR_ARG, "handle already in the batch");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, PAMC_ERR_CUDA, "cudaSetDevice failed");
    // Inside the batch the schedule ring is refilled one step at a time: after
    // step t it holds steps t+1 .. t+16.  Fill the slots of the steps up to
    // host_t + 15 that the member's own stepping has not built yet.
    const pamc_params &p = h->p;
    const int64_t want = std::min<int64_t>(h->host_t + kSchedSlots, p.steps);
    if (p.sweeps > 0 && h->sched_end < want) {
        launch_schedule(h->n, h->d_rp, h->d_adj, p.seed, (int32_t)h->sched_end, (int32_t)(want - h->sched_end),
                        p.sweeps, 0, kSchedSlots, h->d_order, h->d_lvl, h->d_nlev, h->d_skey, h->d_scnt,
                        h->stream, h->d_ell, h->ell_w, h->d_pos);
        h->launches += 1;
        h->sched_end = want;
    }
    // no re-draw is pending when the member joins (a single run re-draws by
    // step index and leaves the batch's flag as its last restart set it)
    cudaError_t e = cudaMemsetAsync(reinterpret_cast<char *>(h->d_ctl) + offsetof(DevCtl, redraw), 0, sizeof(int32_t),
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bfail(b, PAMC_ERR_CUDA, "member sync: %s", cudaGetErrorString(e));
    b->members.push_back(h);
    b->dirty = true;
    return PAMC_OK;
}

pamc_status pamc_batch_step(pamc_batch b, int32_t nsteps) {
    PAMC_RANGE("pamc_batch_step");
    if (!b || nsteps < 0) return bfail(b, PAMC_ERR_ARG, "null batch or nsteps < 0");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, PAMC_ERR_CUDA, "cudaSetDevice failed");
    for (int32_t it = 0; it < nsteps; ++it) {
        if (b->dirty) {
            const pamc_status s = rebuild(b);
            if (s != PAMC_OK) return s;
        }
        if (!b->exec) break;   // nothing left to run
        const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess) return bfail(b, PAMC_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
        b->launches += b->graph_launches;
        bool finished = false;
        for (pamc_handle h : b->members) {
            if (h->host_t >= h->p.steps) continue;
            h->host_t += 1;
            h->sched_end = std::min<int64_t>(h->host_t + kSchedSlots, h->p.steps);
            h->launches += b->graph_launches;
            finished |= h->host_t >= h->p.steps;
        }
        // a member that finished stays a no-op until the graph is rebuilt;
        // rebuild once every member has finished so the loop ends
        bool any = false;
        for (pamc_handle h : b->members) any |= h->host_t < h->p.steps;
        if (finished && !any) b->dirty = true;
    }
    return PAMC_OK;
}

int32_t pamc_batch_retire(pamc_batch b, pamc_handle *out, int32_t max_out) {
    if (!b || (max_out > 0 && !out)) return -1;
    std::vector<pamc_handle> keep, done;
    for (pamc_handle h : b->members) {
        if (h->host_t >= h->p.steps && (int32_t)done.size() < max_out) done.push_back(h);
        else keep.push_back(h);
    }
    if (!done.empty()) {
        if (cudaSetDevice(b->device) != cudaSuccess) return -1;
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return -1;
        for (size_t i = 0; i < done.size(); ++i) out[i] = done[i];
        b->members.swap(keep);
        b->dirty = true;
    }
    return (int32_t)done.size();
}

int pamc_size_class(int32_t n) { return batch_class(n); }

pamc_status pamc_batch_set_shape(pamc_batch b, int size_class, int groups_per_cta, int warps_per_group) {
    if (!b) return bfail(b, PAMC_ERR_ARG, "null batch");
    if (size_class < 0 || size_class >= kClasses) return bfail(b, PAMC_ERR_ARG, "size class must be 0, 1 or 2");
    if (groups_per_cta < 1 || warps_per_group < 1 || groups_per_cta * warps_per_group > 32)
        return bfail(b, PAMC_ERR_ARG, "need groups >= 1, warps >= 1 and groups * warps <= 32");
    b->shape[size_class].groups_per_cta = groups_per_cta;
    b->shape[size_class].warps_per_group = warps_per_group;
    b->dirty = true;
    return PAMC_OK;
}

pamc_status pamc_batch_set_lanes(pamc_batch b, int size_class, int lanes_per_vertex) {
    if (!b) return bfail(b, PAMC_ERR_ARG, "null batch");
    if (size_class < 0 || size_class >= kClasses) return bfail(b, PAMC_ERR_ARG, "size class must be 0, 1 or 2");
    if (!batch_lanes_ok(lanes_per_vertex)) return bfail(b, PAMC_ERR_ARG, "lanes per vertex must be 1, 2 or 4");
    b->shape[size_class].lanes_per_vertex = lanes_per_vertex;
    b->dirty = true;
    return PAMC_OK;
}

pamc_status pamc_batch_set_placement(pamc_batch b, int size_class, int global_spins) {
    if (!b || size_class < 0 || size_class >= kClasses) return bfail(b, PAMC_ERR_ARG, "bad batch or size class");
    b->global[size_class] = global_spins != 0;
    b->dirty = true;
    return PAMC_OK;
}

pamc_status pamc_batch_get_placement(pamc_batch b, int size_class, int *global_spins) {
    if (!b || !global_spins || size_class < 0 || size_class >= kClasses)
        return bfail(b, PAMC_ERR_ARG, "bad batch, size class or null argument");
    *global_spins = b->global[size_class] ? 1 : 0;
    return PAMC_OK;
}

pamc_status pamc_batch_get_lanes(pamc_batch b, int size_class, int *lanes_per_vertex) {
    if (!b || !lanes_per_vertex) return bfail(b, PAMC_ERR_ARG, "null argument");
    if (size_class < 0 || size_class >= kClasses) return bfail(b, PAMC_ERR_ARG, "size class must be 0, 1 or 2");
    *lanes_per_vertex = b->shape[size_class].lanes_per_vertex;
    return PAMC_OK;
}

pamc_status pamc_batch_get_shape(pamc_batch b, int size_class, int *groups_per_cta, int *warps_per_group) {
    if (!b || !groups_per_cta || !warps_per_group) return bfail(b, PAMC_ERR_ARG, "null argument");
    if (size_class < 0 || size_class >= kClasses) return bfail(b, PAMC_ERR_ARG, "size class must be 0, 1 or 2");
    *groups_per_cta = b->shape[size_class].groups_per_cta;
    *warps_per_group = b->shape[size_class].warps_per_group;
    return PAMC_OK;
}

int32_t pamc_batch_size(pamc_batch b) { return b ? (int32_t)b->members.size() : 0; }

int32_t pamc_batch_active(pamc_batch b) {
    if (!b) return 0;
    int32_t a = 0;
    for (pamc_handle h : b->members) a += h->host_t < h->p.steps;
    return a;
}

int64_t pamc_batch_launch_count(pamc_batch b) { return b ? b->launches : 0; }

int64_t pamc_batch_graph_builds(pamc_batch b) { return b ? b->rebuilds : 0; }

pamc_status pamc_batch_sync(pamc_batch b) {
    if (!b) return PAMC_ERR_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, PAMC_ERR_CUDA, "cudaSetDevice failed");
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, PAMC_ERR_CUDA, "batch sync: %s", cudaGetErrorString(e));
    return PAMC_OK;
}

pamc_status pamc_batch_last_error(pamc_batch b, char *buf, size_t len) {
    if (!buf || len == 0) return PAMC_ERR_ARG;
    snprintf(buf, len, "%s", b ? b->err : g_create_err);
    return PAMC_OK;
}

void pamc_batch_destroy(pamc_batch b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (DevBuf *d : {&b->sw, &b->swi, &b->sd, &b->sdi, &b->prep, &b->tabs, &b->ctl, &b->ncm, &b->ncmi, &b->rd,
                      &b->rdi})
        if (d->p) cudaFree(d->p);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
