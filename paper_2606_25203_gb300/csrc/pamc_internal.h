// pamc_internal.h -- device data layout and kernel entry points of libpamc.
#pragma once
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <vector>

#include "../../include/pamc.h"
#include "pamc_device.cuh"

namespace pamc {

constexpr int kHistMax = 64;   // longest stagnation window supported
// Populations up to this size run the population step in one CTA (prefix
// sums and the NCM target sort in shared memory); larger ones (up to
// kMaxPopulation) in several kernels with the prefix sums in device memory.
constexpr int32_t kPrepOneCtaMaxR = 16384;
constexpr int32_t kMaxPopulation = 1 << 20;
constexpr int32_t kNcmSelectMaxTop = 16384;   // NCM targets sorted in one CTA's shared memory

// Algorithm 1's controller state, resident in device memory so that a whole
// iteration (resample, NCM, sweeps, M*, control) runs without the host.
struct DevCtl {
    int32_t t;            // global iteration index (keys the random streams)
    int32_t z, cycle, cooldown, enable_cm, done;
    int32_t ncm_last;     // NCM applied in the last iteration
    int32_t hist_len;
    int32_t resampled;    // the current iteration resampled (z > 1)
    int32_t ncm_active;   // the current iteration applies NCM
    int32_t restart;      // the last iteration restarted (reinit pending)
    int32_t err;          // device-side error code (pamc_status), 0 = none
    int32_t best_replica; // replica holding M* when it was last improved
    int32_t best_owned;   // the replica holding M* is one of this handle's own (always, unless the
                          // population is split over processes)
    int32_t redraw;       // a restart re-draw pending for a batch member (raised by the controller)
    int32_t pad_;
    double beta, delta, dbeta;
    int64_t mstar;        // best cut so far (INT64_MIN = none yet)
    int64_t ncm_flipped, ncm_dE_max;
    int64_t hist[kHistMax];
    // dense sweeps: coupling rows gathered by the field update (positions
    // that flipped in some replica) and positions visited, since pamc_init
    int64_t dense_rows, dense_positions;
    // sparse Ising sweeps: replica spins that changed at a visit, since pamc_init
    int64_t sweep_flips;
};

// Per-(t, sweep) update schedule: the random order's dependency levels.
// order[] lists the vertices level by level; lvl_ptr[l]..lvl_ptr[l+1] is
// level l.  No two vertices of one level are coupled, and every coupled
// pair is ordered exactly as in the random permutation.
struct SchedView {
    const int32_t *order;    // [slots][S][n]: k | deg_k << 24
    const int32_t *lvl_ptr;  // [slots][S][n+1]
    const int32_t *nlev;     // [slots][S]
    const uint32_t *ell;     // [slots][S][ceil(n/32)*32*W] or nullptr (CSR reads)
    const int2 *pos;         // [slots][S][n]: {k | deg << 24, sum_j J_kj} (with ell)
    int32_t W;               // ELL width (a multiple of 4, zero-padded)
    // per vertex {M1 * 0x11111111, M2 * 0x11111111, H - sum_j |J_kj|, 0}
    // (M1, M2: the weight of the negative couplings in ELL slots 0..7 and
    // 8..15): the biased 4-bit lanes of sweep_nibble.cu, or nullptr
    const int4 *nibc = nullptr;
};

// Everything the Ising sweep of one instance needs (single or batched launch).
struct SweepDesc {
    const int32_t *rp;
    const uint32_t *adj;
    const int32_t *sorder, *slvl, *snlev;
    const uint32_t *sell;
    const int2 *spos;
    const uint64_t *tab;
    const int8_t *src;
    const int32_t *parent;
    const int8_t *ncm_buf;
    const int32_t *ncm_idx;
    int8_t *dst;
    int64_t *E_dst;
    const DevCtl *ctl;
    int32_t n, n_pad, H, R, S, t, slot, W;
    PhiloxKeys K;
    // batched launches: the step index comes from ctl->t, which selects the
    // double-buffered spins/energies and the schedule slot; steps >= t_end are no-ops
    int8_t *sp[2];
    int64_t *en[2];
    int32_t slots, t_end;
    int32_t push;   // push-model sweep (H <= 63, ELL, one lane per vertex, S >= 1)
    int64_t Wsum;   // Potts: sum_{i<j} w_ij (E = -sum_k syn_sigma_k(k) - W)
    uint32_t *gsp;  // Ising: the groups' spin words in device memory (n_pad words a group), or nullptr
    int32_t gbase;  // group index of the first local group in the whole population (keys the draws)
    const int4 *nibc;   // biased 4-bit lanes: the per-vertex constants (SchedView::nibc), or nullptr
};

struct SchedDesc {
    const int32_t *rp;
    const uint32_t *adj;
    int32_t *order, *lvl, *nlev, *scnt;
    uint32_t *skey, *ell;
    int2 *pos;
    int32_t n, t0, S, slots, W;
    uint32_t key0, key1;
    // batched launches (ctl != nullptr): after step t's controller ran, build
    // the schedule of step ctl->t + ahead, unless it is >= t_end or ctl->done
    const DevCtl *ctl;
    int32_t ahead, t_end;
};

struct PrepDesc {
    const int64_t *E_src;
    DevCtl *ctl;
    int32_t *parent, *count, *ncm_idx, *targets;
    int32_t R, kind, do_resample, n_top, tau;
    uint32_t key0, key1;
    const int64_t *en[2];   // E_src = en[ctl->t & 1]
    int32_t t_end;
    int32_t *fam;           // [2][R] lineage, double-buffered by step parity
    int32_t fam_reset;      // a restart re-initialises the population
};

struct TabDesc {
    const DevCtl *ctl;
    uint64_t *tab;
    int32_t rule, H, t_end;
    int32_t kind;   // 0 Ising (2H+1 thresholds), 1 Potts cascaded (T1 over (4H+1)^2, then T2)
};

struct CtlDesc {
    const int64_t *E;
    const int8_t *spins;
    int8_t *best;
    DevCtl *ctl;
    int64_t W, target;
    double reheat, beta0;
    int32_t n, R, stagnation, z_rst, win_short, win_long, max_ds, max_dl;
    const int64_t *en[2];   // E = en[(ctl->t + 1) & 1], spins = sp[(ctl->t + 1) & 1]
    const int8_t *sp[2];
    int32_t t_end;
};

// Batched cluster moves (members with stagnation control, Max-Cut): items
// (member, target q).
struct NcmDesc {
    const int32_t *rp;
    const uint32_t *adj;
    const int32_t *parent, *targets;
    int8_t *ncm_buf;
    uint32_t *nkey;
    DevCtl *ctl;
    const int8_t *sp[2];
    const int64_t *en[2];
    int32_t n, R, n_top, trials, t_end;
    uint32_t key0, key1;
};

// Batched restart re-draws (members with restart_reinit).
constexpr int kRedrawPerThread = 16;   // spin-draw elements (group, vertex) per thread of a re-draw item
struct RedrawDesc {
    const int32_t *rp;
    const uint32_t *adj;
    DevCtl *ctl;
    int8_t *sp[2];
    int64_t *en[2];
    int64_t Wsum;
    int32_t n, R, kind, K;
    uint32_t key0, key1;
};
cudaError_t launch_ncm_batched(const NcmDesc *descs, const int2 *items, int32_t nitems, int32_t n_max,
                               cudaStream_t st);
cudaError_t launch_redraw_batched(const RedrawDesc *descs, int32_t nmem, const int2 *spin_items, int32_t nspin,
                                  const int2 *energy_items, int32_t nenergy, cudaStream_t st);

// Allows every launch of `func` with up to `bytes` of dynamic shared memory
// by raising the kernel's limit to the device's opt-in maximum (minus its
// static shared memory).  The limit is never lowered, so launches enqueued or
// captured into a graph earlier with a larger size stay valid whatever the
// order of later launches.
template <typename F>
inline cudaError_t allow_dynamic_smem(F *func, size_t bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, func);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int lim = optin - (int)a.sharedSizeBytes;
    if ((long long)bytes > (long long)lim) return cudaErrorInvalidValue;
    if (a.maxDynamicSharedSizeBytes >= lim) return cudaSuccess;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

// Launch configuration of the sparse sweep kernel.
struct SweepCfg {
    int groups_per_cta;   // replica groups in one CTA
    int warps_per_group;  // warps cooperating on one group's level
    int lanes_per_vertex = 1;  // Ising, ELL: lanes sharing one vertex's couplings (1, 2, 4, .., 32)
};

// Builds the (t, sweep) schedules of nt steps starting at t0 into ring slots
// t % slots.  order[i] = k | deg_k << 24.  With ell != nullptr the nonzero
// couplings of position i are also written position-indexed (ELL of width W,
// W >= the largest degree).
void launch_schedule(int32_t n, const int32_t *rp, const uint32_t *adj, uint64_t seed, int32_t t0,
                     int32_t nt, int32_t S, int32_t slot0, int32_t slots, int32_t *order,
                     int32_t *lvl_ptr, int32_t *nlev, uint32_t *skey, int32_t *scnt,
                     cudaStream_t st, uint32_t *ell = nullptr, int32_t W = 0,
                     int2 *pos = nullptr);

// Dynamic shared memory of the Ising sweep; with global_spins the groups'
// spin words live in device memory instead (see SweepDesc::gsp).
size_t sweep_ising_smem_bytes(int32_t n, int32_t H, SweepCfg cfg, bool global_spins = false);
// Push-model Ising sweeps (fields kept in shared memory, updated on flips):
// used where H <= 63, on ELL schedules with one lane per vertex and S >= 1,
// when the environment variable PAMC_SWEEP_PUSH is "1".
bool sweep_push_enabled();
bool sweep_push_ok(int32_t H, int32_t S, bool ell, int lanes_per_vertex);
void launch_schedule_batched(const SchedDesc *descs, const int2 *items, int32_t nitems, int32_t n_max,
                             cudaStream_t st);
cudaError_t launch_population_batched(const PrepDesc *prep, const TabDesc *tabs, int32_t ninst,
                                      int32_t R_max, cudaStream_t st);
cudaError_t launch_control_batched(const CtlDesc *descs, int32_t ninst, cudaStream_t st);
size_t prep_smem_bytes(int32_t R);
cudaError_t launch_sweep_ising_batched(int rule, bool ell, const SweepDesc *descs, const int2 *items,
                                       int32_t nitems, int32_t n_max, SweepCfg cfg, cudaStream_t st,
                                       bool global_spins = false);
// Batched three-state Potts sweeps (cascaded sampler), one launch per (ELL, size class).
cudaError_t launch_sweep_potts_batched(bool ell, const SweepDesc *descs, const int2 *items, int32_t nitems,
                                       int32_t n_max, SweepCfg cfg, cudaStream_t st);
cudaError_t launch_sweep_ising(int rule, int32_t n, const int32_t *rp, const uint32_t *adj,
                               int32_t H, const pamc_params &p, int32_t t, int32_t slot,
                               SchedView sv, const uint64_t *tab, const int8_t *src,
                               const int32_t *parent, const int8_t *ncm_buf,
                               const int32_t *ncm_idx, int8_t *dst, int64_t *E_dst,
                               const DevCtl *ctl, SweepCfg cfg, cudaStream_t st, uint32_t *gsp = nullptr,
                               int32_t rbase = 0);

// Ising sweeps with 16-bit field lanes (sweep_wide.cu): instances with
// 127 < H <= 32767; two words per vertex and replica group (8n bytes), in
// shared memory or, with gsp, in device memory (2 * n_pad words a group).
constexpr int32_t kByteLaneMaxH = 127;
constexpr int32_t kWideLaneMaxH = 32767;
size_t sweep_wide_smem_bytes(int32_t n, SweepCfg cfg, bool global_spins);
cudaError_t launch_sweep_ising_wide(int rule, int32_t n, const int32_t *rp, const uint32_t *adj, int32_t H,
                                    const pamc_params &p, int32_t t, int32_t slot, SchedView sv,
                                    const uint64_t *tab, const int8_t *src, const int32_t *parent,
                                    const int8_t *ncm_buf, const int32_t *ncm_idx, int8_t *dst, int64_t *E_dst,
                                    const DevCtl *ctl, SweepCfg cfg, cudaStream_t st, uint32_t *gsp,
                                    int32_t rbase = 0);

// Ising sweeps with 4-bit field lanes, eight replicas per word
// (sweep_nibble.cu), S >= 1, one lane per vertex, words in shared memory; off
// with PAMC_SWEEP_NIBBLE=0.  Groups of eight replicas (ceil(R / 8) of them).
// Fixed bias: H <= 7 on ELL rows of width 4 or 8.  Biased lanes (per-vertex
// constants, two accumulators): ELL width 4 to 16 with sum |J| <= 15 over
// the slots 0..7 and over the slots 8..15 of every vertex.
constexpr int32_t kNibbleMaxH = 7;
constexpr int32_t kNibbleHalfMaxH = 15;
constexpr int32_t kNibbleBiasedMaxH = 2 * kNibbleHalfMaxH;
bool sweep_nibble_enabled();
bool sweep_nibble_ok(int32_t H, int32_t S, int32_t ell_w, int lanes_per_vertex, bool global_spins,
                     bool biased_ok);
// The biased lanes' per-vertex constants from the packed CSR (J in the top
// byte, the ELL slot order: the nonzero couplings in CSR order); false when
// some vertex exceeds kNibbleHalfMaxH in a half or the width exceeds 16.
bool nibble_biased_constants(int32_t n, const int32_t *rp, const uint32_t *adj, int32_t H, int32_t ell_w,
                             std::vector<int4> &out);
size_t sweep_nibble_smem_bytes(int32_t n, int32_t H, SweepCfg cfg);
cudaError_t launch_sweep_ising_nib(int rule, int32_t n, int32_t H, const pamc_params &p, int32_t t, int32_t slot,
                                   SchedView sv, const uint64_t *tab, const int8_t *src, const int32_t *parent,
                                   const int8_t *ncm_buf, const int32_t *ncm_idx, int8_t *dst, int64_t *E_dst,
                                   const DevCtl *ctl, SweepCfg cfg, cudaStream_t st, int32_t rbase);
// Batched 4-bit-lane sweeps (members as for the single launch, fixed or
// biased lanes per member, words on chip); items (member, block of groups of
// eight).
cudaError_t launch_sweep_ising_nib_batched(int rule, bool biased, const SweepDesc *descs, const int2 *items,
                                           int32_t nitems, int32_t n_max, SweepCfg cfg, cudaStream_t st);

// Sweep kinds: 0 Ising, 1 Potts K=3 cascaded sampler, 2 Potts softmax noisy argmax;
// every kind keeps groups of four replicas.
size_t sweep_smem_bytes(int kind, int32_t n, int32_t H, SweepCfg cfg);
size_t sweep_softmax_smem_bytes(int32_t n, int32_t H, SweepCfg cfg);
size_t sweep_potts_smem_bytes(int32_t n, int32_t H, SweepCfg cfg);
cudaError_t launch_sweep_potts(int32_t n, const int32_t *rp, const uint32_t *adj, int32_t H, const pamc_params &p,
                               int32_t t, int32_t slot, SchedView sv, const uint64_t *tab, const int8_t *src,
                               const int32_t *parent, int8_t *dst, int64_t *E_dst, const DevCtl *ctl,
                               SweepCfg cfg, int64_t Wsum, cudaStream_t st, int32_t rbase = 0);
cudaError_t launch_sweep_softmax(int32_t n, const int32_t *rp, const uint32_t *adj, int32_t H,
                                 const pamc_params &p, int32_t t, int32_t slot, SchedView sv,
                                 const uint64_t *tab, const int8_t *src, const int32_t *parent,
                                 const int32_t *ncm_idx, int8_t *dst, int64_t *E_dst, const DevCtl *ctl,
                                 SweepCfg cfg, int64_t Wsum, cudaStream_t st, int32_t rbase = 0);

// rbase: index of the first local replica in the whole population (a
// multiple of 4; nonzero when the population is split over processes): the
// random draws are keyed by the replica's index in the whole population.
cudaError_t launch_sweep(int kind, int rule, int32_t n, const int32_t *rp, const uint32_t *adj,
                         int32_t H, const pamc_params &p, int32_t t, int32_t slot, SchedView sv,
                         const uint64_t *tab, const int8_t *src, const int32_t *parent,
                         const int8_t *ncm_buf, const int32_t *ncm_idx, int8_t *dst,
                         int64_t *E_dst, const DevCtl *ctl, SweepCfg cfg, int64_t Wsum,
                         cudaStream_t st, uint32_t *gsp = nullptr, int32_t rbase = 0, bool nib = false);

// Random (re)initialisation of the population with key t, and its energies;
// when only_if_restart is set the kernels do nothing unless the controller
// has just restarted the schedule.
cudaError_t launch_init(int kind, int32_t K, int32_t n, const int32_t *rp, const uint32_t *adj, int32_t R,
                        uint64_t seed, int32_t t, int only_if_restart, const DevCtl *ctl,
                        int64_t Wsum, int8_t *spins, int64_t *E, cudaStream_t st, int32_t rbase = 0);

// Energies of a given population from the definition (one CTA per replica).
cudaError_t launch_energy(int kind, int32_t n, const int32_t *rp, const uint32_t *adj, int32_t R,
                          const DevCtl *ctl, int64_t Wsum, const int8_t *spins, int64_t *E, cudaStream_t st);

// ---- a population split over processes (shard.cu): rows[i] of src -> row i of dst
cudaError_t launch_gather_rows(int32_t n, const int32_t *rows, int32_t nrows, const int8_t *src, int8_t *dst,
                               cudaStream_t st);

// ---- diagnostics (diag.cu)
// Pairwise corrected Hamming distances of a +-1 population (R rows of n int8):
// hist[min(d, n - d)] += 1 and *sum += min(d, n - d) over all pairs r < r'.
// bits: scratch of R * ceil(n / 32) words.  hist and sum are zeroed first.
cudaError_t launch_hamming(int32_t n, int32_t R, const int8_t *spins, uint32_t *bits,
                           unsigned long long *hist, unsigned long long *sum, cudaStream_t st);
// The same on the tensor cores: the e4m3 population (scratch of
// hamming_tc_scratch bytes) and its overlaps S S^T by tcgen05 (err: the
// device status word, PAMC_ERR_TIMEOUT if a bounded wait gives up).
bool hamming_tc_enabled(int32_t n, int32_t R);
size_t hamming_tc_scratch(int32_t n, int32_t R);
cudaError_t launch_hamming_tc(int32_t n, int32_t R, const int8_t *spins, uint8_t *Sb, unsigned long long *hist,
                              unsigned long long *sum, int *err, cudaStream_t st);

// ---- dense instances (dense.cu)
cudaError_t launch_dense_validate(int32_t n, const int8_t *J, int *err, cudaStream_t st);
cudaError_t launch_dense_negate_sum(size_t total, int8_t *J, unsigned long long *wsum, cudaStream_t st);
cudaError_t launch_dense_perm(int32_t n, uint64_t seed, int32_t t, int32_t S, int32_t *perm,
                              uint32_t *skey, int32_t *sidx, int32_t *boff, const DevCtl *ctl, cudaStream_t st);
size_t dense_perm_offsets(int32_t S);   // int32 bucket offsets launch_dense_perm needs
cudaError_t launch_dense_tables(int rule, int32_t Hc, int32_t n, DevCtl *ctl, uint64_t *tab,
                                cudaStream_t st);
size_t dense_recompute_smem();
cudaError_t launch_dense_recompute(int32_t n, int32_t R, const int8_t *J, const int8_t *src,
                                   const int32_t *parent, const int8_t *ncm_buf,
                                   const int32_t *ncm_idx, int32_t *H, const DevCtl *ctl,
                                   cudaStream_t st, int restart_t);
cudaError_t launch_dense_energy(int32_t n, int32_t R, const int32_t *H, const int8_t *spins, int64_t *E,
                                const DevCtl *ctl, cudaStream_t st, int restart_t);
cudaError_t launch_init_spins(int kind, int32_t K, int32_t n, int32_t R, uint64_t seed, int32_t t,
                              int only_if_restart, const DevCtl *ctl, int8_t *spins, cudaStream_t st,
                              int32_t rbase = 0);
int dense_block_positions();
int dense_sweep_threads();
size_t dense_sweep_smem(int32_t n, int32_t R, int32_t rows_per, bool tcu);
cudaError_t launch_dense_sweep(int32_t n, int32_t R, int32_t S, int32_t rule, int32_t Hc, int32_t t,
                               uint64_t seed, int32_t n_upd, int32_t rows_per, int32_t grid,
                               const int8_t *J, const int32_t *perm, const uint64_t *tab,
                               const int8_t *src, const int32_t *parent, const int8_t *ncm_buf,
                               const int32_t *ncm_idx, int32_t *H, int8_t *dst, int64_t *E,
                               int32_t *G, uint32_t *T, uint32_t *T2, unsigned long long *flip,
                               unsigned long long *snew, void *bar, DevCtl *ctl, cudaStream_t st, bool tcu,
                               int32_t rbase = 0);
cudaError_t launch_dense_to_e4m3(size_t total, int8_t *J, cudaStream_t st);

// ---- dense recompute on tcgen05 (dense_tc.cu), n a multiple of 16
bool dense_tc_supported(int32_t n);
size_t dense_tc_smem();
// map: 128-byte CUtensorMap storage (64-byte aligned)
cudaError_t dense_tc_map(void *map, const void *base, int32_t rows, int32_t cols, int32_t box_rows);
cudaError_t launch_dense_recompute_tc(int32_t n, int32_t R, const void *mapJ, const void *mapS,
                                      const int8_t *src, const int32_t *parent, const int8_t *ncm_buf,
                                      const int32_t *ncm_idx, uint8_t *Sb, int32_t *H, DevCtl *ctl,
                                      cudaStream_t st, int restart_t);

}  // namespace pamc
