// dense_tc.cu -- the full field recompute of the dense instance, H = J S
// (row a4), on the 5th-generation tensor cores.
//
// A CTA owns 256 rows of J.  The K dimension (n couplings) is streamed in
// 128-byte slices: TMA copies the 256 x 128-byte slice of J and the matching
// 64 x 128-byte slice of the population (e4m3 spins, replicas padded to 64)
// into shared memory with the 128-byte swizzle, five slices in flight.  One
// elected thread issues tcgen05.mma kind::f8f6f4 (M=128, N=64, K=32, two M
// tiles, four K steps per slice) into a 128-column fp32 accumulator in tensor
// memory and frees each slice with tcgen05.commit on the slice's mbarrier.
// Four warps read the accumulator back with tcgen05.ld and store the int32
// fields.  Products are +-1 or 0 and partial sums integers below 2^24, so the
// result is the exact field (the same check as the mma.sync recompute).
//
// Every wait is bounded; on expiry the kernel records PAMC_ERR_TIMEOUT, lets
// the copies and MMAs it issued complete (bounded), frees tensor memory and
// returns.
#include <cuda.h>

#include <mutex>

#include "pamc_device.cuh"
#include "pamc_internal.h"
#include "tc_sm100.cuh"

namespace pamc {

namespace {

constexpr int kTcRows = 256;                 // rows of J per CTA (two M=128 tiles)
constexpr int kTcKB = 128;                   // K bytes per slice (one swizzle atom)
constexpr int kTcStages = 5;
constexpr int kTcABytes = kTcRows * kTcKB;   // 32 KB
constexpr int kTcBBytes = 64 * kTcKB;        // 8 KB
constexpr int kTcStageBytes = kTcABytes + kTcBBytes;
constexpr int kTcThreads = 128;
constexpr uint32_t kTcCols = 128;            // tensor memory columns: 2 tiles x N=64

// instruction descriptor: D f32, A and B e4m3, both K-major, N=64, M=128
constexpr uint32_t kTcIdesc = (1u << 4) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// e4m3 population: Sb[r][k] = +-1.0 of replica r's spin k (the slot's parent
// or NCM row), 0 for padding replicas r >= R.  n is a multiple of 16.
__global__ void k_dense_spins_e4m3(int32_t n, int32_t R, const int8_t *__restrict__ src,
                                   const int32_t *__restrict__ parent, const int8_t *__restrict__ ncm_buf,
                                   const int32_t *__restrict__ ncm_idx, uint8_t *__restrict__ Sb,
                                   const DevCtl *__restrict__ ctl, int restart_t) {
    if (restart_t >= 0 ? !(ctl->restart && ctl->t == restart_t) : ctl->done != 0) return;
    const int32_t nc = n / 16;
    const size_t total = (size_t)64 * nc;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)(x / nc), c = (int32_t)(x % nc);
        uint4 o = make_uint4(0u, 0u, 0u, 0u);
        if (r < R) {
            const int32_t qn = ncm_idx[r];
            const int8_t *row = qn >= 0 ? ncm_buf + (size_t)qn * n : src + (size_t)parent[r] * n;
            const uint4 v = *reinterpret_cast<const uint4 *>(row + (size_t)c * 16);
            o.x = (v.x & 0x80808080u) | 0x38383838u;
            o.y = (v.y & 0x80808080u) | 0x38383838u;
            o.z = (v.z & 0x80808080u) | 0x38383838u;
            o.w = (v.w & 0x80808080u) | 0x38383838u;
        }
        *reinterpret_cast<uint4 *>(Sb + (size_t)r * n + (size_t)c * 16) = o;
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_dense_recompute_tc(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmS, int32_t n,
                     int32_t R, int32_t *__restrict__ H, DevCtl *__restrict__ ctl, int restart_t) {
    if (restart_t >= 0 ? !(ctl->restart && ctl->t == restart_t) : ctl->done != 0) return;
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;
    uint8_t *base = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t row0 = blockIdx.x * kTcRows;
    const int32_t nk = (n + kTcKB - 1) / kTcKB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(&done, 1);
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // producer: slice kc into stage kc % kTcStages once the MMAs of its
        // previous use have completed
        int32_t issued = 0;
        for (int32_t kc = 0; kc < nk; ++kc) {
            const int s = kc % kTcStages;
            const int32_t round = kc / kTcStages;
            if (round > 0 && !mbar_wait(&empty[s], (uint32_t)((round - 1) & 1))) {
                atomicCAS(&ctl->err, 0, (int)PAMC_ERR_TIMEOUT);
                s_err = 1;
                break;
            }
            if (*(volatile int *)&s_err) break;
            uint8_t *A = base + (size_t)s * kTcStageBytes;
            mbar_expect_tx(&full[s], (uint32_t)kTcStageBytes);
            tma_load_2d(A, &tmJ, kc * kTcKB, row0, &full[s]);
            tma_load_2d(A + kTcABytes, &tmS, kc * kTcKB, 0, &full[s]);
            issued = kc + 1;
        }
        // every issued slice has landed before the CTA may leave (bounded)
        for (int32_t kc = (issued > kTcStages ? issued - kTcStages : 0); kc < issued; ++kc)
            mbar_wait(&full[kc % kTcStages], (uint32_t)((kc / kTcStages) & 1));
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int32_t kc = 0; kc < nk; ++kc) {
            const int s = kc % kTcStages;
            if (!mbar_wait(&full[s], (uint32_t)((kc / kTcStages) & 1)) || *(volatile int *)&s_err) {
                atomicCAS(&ctl->err, 0, (int)PAMC_ERR_TIMEOUT);
                s_err = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(base + (size_t)s * kTcStageBytes);
            const uint32_t b0 = a0 + kTcABytes;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int ks = 0; ks < kTcKB / 32; ++ks)
                    tc_mma(tmem + (uint32_t)(mt * 64), sw128_desc(a0 + mt * 128 * kTcKB) + (uint64_t)(2 * ks),
                           sw128_desc(b0) + (uint64_t)(2 * ks), kTcIdesc, (kc > 0 || ks > 0) ? 1u : 0u);
            tc_commit(&empty[s]);
        }
        tc_commit(&done);   // completes once every MMA issued above has completed
    }
    __syncwarp();
    // epilogue: warp w holds rows 32w .. 32w+31 of each M tile in its lanes
    const bool ok = mbar_wait(&done, 0u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && !*(volatile int *)&s_err) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int32_t row = row0 + mt * 128 + warp * 32 + lane;
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                uint32_t v[16];
                tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * 64 + c0), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int r = c0 + j;
                    if (row < n && r < R) H[(size_t)r * n + row] = __float2int_rn(__uint_as_float(v[j]));
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicCAS(&ctl->err, 0, (int)PAMC_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

}  // namespace

bool dense_tc_supported(int32_t n) { return n >= 16 && n % 16 == 0 && encode_fn() != nullptr; }

size_t dense_tc_smem() { return (size_t)kTcStages * kTcStageBytes + 1024; }

// 2-D map over a row-major byte matrix of `rows` rows of `cols` bytes
// (cols a multiple of 16), box `box_rows` x 128 bytes, 128-byte swizzle.
cudaError_t dense_tc_map(void *map, const void *base, int32_t rows, int32_t cols, int32_t box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || cols % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols};
    const cuuint32_t box[2] = {(cuuint32_t)kTcKB, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(reinterpret_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                          const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_dense_recompute_tc(int32_t n, int32_t R, const void *mapJ, const void *mapS,
                                      const int8_t *src, const int32_t *parent, const int8_t *ncm_buf,
                                      const int32_t *ncm_idx, uint8_t *Sb, int32_t *H, DevCtl *ctl,
                                      cudaStream_t st, int restart_t) {
    if (R > 64 || n % 16 != 0) return cudaErrorInvalidValue;
    const size_t chunks = (size_t)64 * (n / 16);
    int grid = (int)((chunks + 255) / 256);
    if (grid > 152 * 8) grid = 152 * 8;
    k_dense_spins_e4m3<<<grid, 256, 0, st>>>(n, R, src, parent, ncm_buf, ncm_idx, Sb, ctl, restart_t);
    const size_t smem = dense_tc_smem();
    cudaError_t e = allow_dynamic_smem(k_dense_recompute_tc, smem);
    if (e != cudaSuccess) return e;
    const CUtensorMap *mj = reinterpret_cast<const CUtensorMap *>(mapJ);
    const CUtensorMap *ms = reinterpret_cast<const CUtensorMap *>(mapS);
    k_dense_recompute_tc<<<(n + kTcRows - 1) / kTcRows, kTcThreads, smem, st>>>(*mj, *ms, n, R, H, ctl, restart_t);
    return cudaGetLastError();
}

}  // namespace pamc
