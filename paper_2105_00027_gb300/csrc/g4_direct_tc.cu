// Direct term of the particle-hole magnetic G4 update on the tcgen05 tensor
// cores:
//   Dir(K1, K2, Q) = sum_r a_r(K1) b_r(K2),
//   a_r(K1) = s_r sum_s s G_s(K1+Q, K1),  b_r(K2) = sum_s s G_s(K2, K2+Q).
// For fixed Q this is a sum of rank-1 outer products over the batch: a GEMM
// whose K dimension is the batch (the paper's accumulation, Eq. (1), Sec. 2.1,
// in the particle-hole magnetic channel).
//
// Operands come from k_pack_direct: K-major rows of TF32 values, the complex
// product embedded as real products (Re|Im halves along K), each operand split
// x = hi + lo.  One output tile is 128 rows K2 x 128 columns K1 of one Q (the
// transposed product, so that tensor-memory lanes -- one thread each in the
// epilogue -- run along K2 and a warp's accumulator accesses stay within a
// 150 KB span); the accumulator tile in tensor memory holds [Re | Im] =
// 128 x 256 FP32.  Per K step three MMAs (hi.hi + hi.lo + lo.hi) accumulate.
//
// Persistent kernel, one CTA per SM, warp roles:
//   warp 0      TMA producer (2-stage shared-memory ring, 96 KB per stage)
//   warp 1      MMA issuer (single thread), two TMEM accumulators (2 x 256 cols)
//   warps 2..9  epilogue: tcgen05.ld -> the direct accumulator
//               accd[Q][K1][K2] += Dir: for one column K1 the 32 lanes of a
//               warp hold 32 consecutive K2, a 512-byte run that is staged in
//               shared memory and added by an asynchronous bulk reduction
// The tiles of Q = 0 accumulate each 32-element K chunk in its own tensor-memory
// accumulator, added to the FP64 accumulator one after the other: for Q = 0
// the operands hold the coherent G0 part of every measurement (density
// channel, or a spin-split G0), and the tensor cores' FP32 accumulation loses
// about one unit in the last place of the running sum per MMA.
// Every mbarrier wait is bounded; on timeout the CTA records G4_DEV_TIMEOUT in
// the status word, stops issuing work, drains its own copies and returns.
#include <cudaTypedefs.h>

#include <cstdio>

#include "g4_internal.h"
#include "g4_ptx.cuh"

namespace {

using namespace g4ptx;

constexpr int kTileM = 128;          // rows K2 per tile
constexpr int kTileN = 128;          // complex columns K1 per tile (MMA N = 256)
constexpr int kKStage = 32;          // TF32 elements of K per stage (128 B rows)
constexpr int kStages = 2;
constexpr int kAB = kTileM * kKStage * 4;          // 16 KB: one A plane per stage
constexpr int kBB = 2 * kTileN * kKStage * 4;      // 32 KB: one B plane per stage
constexpr int kStageBytes = 2 * kAB + 2 * kBB;     // 96 KB
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kTmemCols = 512;
// Epilogue run buffer per warp: 8 columns K1 x 32 lanes K2 of complex FP64.
constexpr int kRunCols = 8;
constexpr int kRunBytes = kRunCols * 32 * 16;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256 + kEpiWarps * kRunBytes;

struct DParams {
    double2* accd;
    unsigned* status;
    int N, NQ, Nwex, Nw2, Bp;
    int nit, njt, ntiles;
    long long budget;  // clock64 cycles per wait
};

// Instruction descriptor: kind::tf32, M = 128, N = 256 ([Re | Im] columns).
constexpr uint32_t kIdesc = idesc_tf32(kTileM, 2 * kTileN);

struct TileCoord {
    int Q, i0, j0;
};

// Tile order: K1 tiles fastest, then K2 tiles, then Q, so that CTAs running at
// the same time share operand tiles in L2.
__device__ __forceinline__ TileCoord tile_coord(const DParams& P, int t) {
    const int jt = t % P.njt;
    t /= P.njt;
    const int it = t % P.nit;
    const int Q = t / P.nit;
    return TileCoord{Q, it * kTileM, jt * kTileN};
}

// Asynchronous FP64 reduction of a shared-memory run into global memory (the
// add is performed at L2), and the calling thread's bulk-group bookkeeping.
__device__ __forceinline__ void bulk_add_f64(double2* gdst, const double2* ssrc, uint32_t bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_u32(ssrc)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1)
    k_direct_tc(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                DParams P) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + kStages * kStageBytes);
    uint64_t* full = bars;                 // [kStages]
    uint64_t* empty = bars + kStages;      // [kStages]
    uint64_t* tfull = bars + 2 * kStages;  // [2]
    uint64_t* tempty = tfull + 2;          // [2]
    uint64_t* mdone = tempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpiWarps);
        }
        mbar_init(mdone, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int nk = (2 * P.Bp) / kKStage;  // stages of K per tile

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;
            for (int t = blockIdx.x; t < P.ntiles && !*abort_flag; t += gridDim.x) {
                const TileCoord tc = tile_coord(P, t);
                for (int ks = 0; ks < nk; ++ks, ++g) {
                    const int s = g % kStages;
                    const uint32_t ph = (g / kStages) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1, P.budget, abort_flag)) break;
                    uint8_t* st = smem + s * kStageBytes;
                    mbar_expect_tx(&full[s], kStageBytes);
                    const int kx = ks * kKStage;
                    tma_load_3d(st, &tmAh, &full[s], kx, tc.i0, tc.Q);
                    tma_load_3d(st + kAB, &tmAl, &full[s], kx, tc.i0, tc.Q);
                    tma_load_4d(st + 2 * kAB, &tmBh, &full[s], kx, tc.j0, 0, tc.Q);
                    tma_load_4d(st + 2 * kAB + kBB / 2, &tmBh, &full[s], kx, tc.j0, 1, tc.Q);
                    tma_load_4d(st + 2 * kAB + kBB, &tmBl, &full[s], kx, tc.j0, 0, tc.Q);
                    tma_load_4d(st + 2 * kAB + kBB + kBB / 2, &tmBl, &full[s], kx, tc.j0, 1, tc.Q);
                }
            }
            // after an abort, wait (bounded) until the copies already issued have landed
            if (*abort_flag) {
                for (uint32_t k = 0; k < (uint32_t)kStages && k < g; ++k) {
                    const uint32_t gg = g - 1 - k;
                    const long long t0 = clock64();
                    while (!mbar_try(&full[gg % kStages], (gg / kStages) & 1) &&
                           clock64() - t0 < kDrainBudget) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0, tl = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < P.ntiles && !*abort_flag; t += gridDim.x) {
                const bool split = tile_coord(P, t).Q == 0;
                uint32_t d_tmem = 0;
                for (int ks = 0; ks < nk; ++ks, ++g) {
                    if (ks == 0 || split) {
                        const int b = tl & 1;
                        if (!mbar_wait(&tempty[b], ((tl >> 1) & 1) ^ 1, P.budget, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        d_tmem = tmem_base + (uint32_t)(b * 2 * kTileN);
                    }
                    const int s = g % kStages;
                    const uint32_t ph = (g / kStages) & 1;
                    if (!mbar_wait(&full[s], ph, P.budget, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + s * kStageBytes);
#pragma unroll
                    for (int k = 0; k < kKStage / 8; ++k) {
                        const uint32_t off = k * 32;  // 8 TF32 = 32 bytes along K
                        const uint64_t ah = sdesc_k128(st + off), al = sdesc_k128(st + kAB + off);
                        const uint64_t bh = sdesc_k128(st + 2 * kAB + off);
                        const uint64_t bl = sdesc_k128(st + 2 * kAB + kBB + off);
                        mma_tf32(d_tmem, ah, bh, kIdesc, ((split ? 0 : ks) | k) != 0);
                        mma_tf32(d_tmem, ah, bl, kIdesc, 1);
                        mma_tf32(d_tmem, al, bh, kIdesc, 1);
                    }
                    mma_commit(&empty[s]);
                    if (split || ks == nk - 1) {
                        mma_commit(&tfull[tl & 1]);
                        ++tl;
                    }
                }
            }
            // wait (bounded) for every MMA this thread issued before TMEM is freed
            mma_commit(mdone);
            const long long t0 = clock64();
            while (!mbar_try(mdone, 0) && clock64() - t0 < kDrainBudget) {
            }
        }
    } else {
        // epilogue warps: lane quadrant from the warp index, column half from the warp group
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        double2* runbuf = (double2*)(smem + kStages * kStageBytes + 256) + (size_t)(warp - 2) * (kRunBytes / 16);
        uint32_t tl = 0;
        bool live = true;
        for (int t = blockIdx.x; live && t < P.ntiles; t += gridDim.x) {
            const TileCoord tc = tile_coord(P, t);
            const int nsub = tc.Q == 0 ? nk : 1;
            for (int sub = 0; sub < nsub; ++sub, ++tl) {
                const int b = tl & 1;
                const uint32_t tph = (tl >> 1) & 1;
                if (!mbar_wait(&tfull[b], tph, P.budget, abort_flag)) {
                    live = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase =
                    tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * 2 * kTileN);
                // this warp's 32 K2 of a column K1 form one contiguous run of accd;
                // runs of kRunCols columns are staged in shared memory and added
                // with bulk reductions (those of a split tile in a fixed order)
                // entries whose K1 + Q or K2 + Q leaves the frequency grid are
                // structurally zero (a or b vanishes): columns with n1 + m >= Nw2 are
                // skipped and runs end at n2 + m = Nw2 when they lie in one k2 block
                const int K2s = tc.i0 + quad * 32;
                const int mq = tc.Q % P.Nwex;
                int nk2 = min(32, P.N - K2s);
                const int n2s = K2s % P.Nw2;
                if (n2s + nk2 <= P.Nw2) nk2 = max(0, min(nk2, P.Nw2 - mq - n2s));
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    const int c0 = half * 64 + c * 32;
                    float re[32], im[32];
                    tmem_ld32(tbase + c0, re);
                    tmem_ld32(tbase + kTileN + c0, im);
                    tmem_wait_ld();
                    if (c == 1) {
                        // last read of the accumulator: hand it back to the MMA warp
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty[b]);
                    }
#pragma unroll
                    for (int g = 0; g < 32; g += kRunCols) {
                        if (lane < kRunCols) {
                            if (nsub > 1) bulk_wait_all();
                            else bulk_wait_read_all();
                        }
                        __syncwarp();
#pragma unroll
                        for (int jj = 0; jj < kRunCols; ++jj)
                            runbuf[jj * 32 + lane] = make_double2((double)re[g + jj], f32_to_f64(im[g + jj]));
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane < kRunCols) {
                            const int K1 = tc.j0 + c0 + g + lane;
                            if (K1 < P.N && nk2 > 0 && K1 % P.Nw2 + mq < P.Nw2)
                                bulk_add_f64(P.accd + ((size_t)tc.Q * P.N + K1) * P.N + K2s,
                                             runbuf + lane * 32, (uint32_t)(16 * nk2));
                            bulk_commit();
                        }
                    }
                }
                // warm L2 with the accumulator lines of this warp's part of the next
                // tile (32 rows K2 x 64 columns K1: 256 lines of 128 bytes, 8 per lane)
                const int tn = t + gridDim.x;
                if (sub == nsub - 1 && tn < P.ntiles) {
                    const TileCoord nc = tile_coord(P, tn);
                    const int k2w = nc.i0 + quad * 32;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int li = lane + 32 * i;            // line index within the warp's block
                        const int col = nc.j0 + half * 64 + (li >> 2);
                        if (col < P.N && k2w + (li & 3) * 8 < P.N) {
                            const double2* ptr =
                                P.accd + ((size_t)nc.Q * P.N + col) * P.N + k2w + (li & 3) * 8;
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
                        }
                    }
                }
            }
        }
        if (lane < kRunCols) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) atomicOr(P.status, (unsigned)G4_DEV_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(kTmemCols)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

struct DirectMaps {
    CUtensorMap Ah, Al, Bh, Bl;
};

bool encode_maps(g4_ctx* h, DirectMaps& m) {
    auto enc = get_encoder();
    if (!enc) return false;
    const G4Dims& d = h->d;
    const cuuint64_t K = 2 * (cuuint64_t)h->Bp;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    {
        const cuuint64_t dims[3] = {K, (cuuint64_t)d.N, (cuuint64_t)d.NQ};
        const cuuint64_t strides[2] = {K * 4, K * 4 * d.N};
        const cuuint32_t box[3] = {kKStage, kTileM, 1};
        for (int i = 0; i < 2; ++i) {
            CUresult r = enc(i ? &m.Al : &m.Ah, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                             i ? (void*)h->Al : (void*)h->Ah, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return false;
        }
    }
    {
        const cuuint64_t dims[4] = {K, (cuuint64_t)d.N, 2, (cuuint64_t)d.NQ};
        const cuuint64_t strides[3] = {K * 4, K * 4 * d.N, K * 4 * d.N * 2};
        const cuuint32_t box[4] = {kKStage, kTileN, 1, 1};
        for (int i = 0; i < 2; ++i) {
            CUresult r = enc(i ? &m.Bl : &m.Bh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                             i ? (void*)h->Bl : (void*)h->Bh, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return false;
        }
    }
    return true;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

}  // namespace

g4_status direct_prepare(g4_ctx* h) {
    DirectMaps* m = new (std::nothrow) DirectMaps();
    if (!m) return g4_fail(h, G4_ERR_OOM, "host allocation of tensor maps");
    if (!encode_maps(h, *m)) {
        delete m;
        return g4_fail(h, G4_ERR_CUDA, "cuTensorMapEncodeTiled failed for the direct-term operands");
    }
    h->tmap_dev = m;
    cudaError_t e = cudaFuncSetAttribute(k_direct_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "direct smem attribute");
    return G4_OK;
}

g4_status direct_run(g4_ctx* h, int) {
    const DirectMaps* m = (const DirectMaps*)h->tmap_dev;
    DParams P;
    P.accd = h->accd;
    P.status = h->dstatus;
    P.N = h->d.N;
    P.NQ = h->d.NQ;
    P.Nwex = h->d.Nwex;
    P.Nw2 = h->d.Nw2;
    P.Bp = h->Bp;
    P.nit = (h->d.N + kTileM - 1) / kTileM;
    P.njt = (h->d.N + kTileN - 1) / kTileN;
    P.ntiles = h->d.NQ * P.nit * P.njt;
    P.budget = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : 4000000000LL;
    const int grid = P.ntiles < sm_count() ? P.ntiles : sm_count();
    k_direct_tc<<<grid, kThreads, kSmemBytes, h->stream>>>(m->Ah, m->Al, m->Bh, m->Bl, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "direct launch");
    return G4_OK;
}

void direct_release(g4_ctx* h) {
    delete (DirectMaps*)h->tmap_dev;
    h->tmap_dev = nullptr;
}
