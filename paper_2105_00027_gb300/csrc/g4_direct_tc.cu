// Direct term of the G4 update on the tcgen05 tensor cores, for the channels
// that have one (particle-hole magnetic and density):
//   Dir(K1, K2, Q) = sum_r a_r(K1) b_r(K2),
//   a_r(K1) = sum_s w_s G~_s(K1+Q, K1),  b_r(K2) = sum_s w_s G~_s(K2, K2+Q)
// (w_s = s for the magnetic channel, 1 for the density channel; G~ = sqrt(s_r) G
// as staged by the G build, so that a_r b_r carries the sign s_r).  For a fixed
// transfer Q this is a sum of rank-1 outer products over the measurements: a
// GEMM whose K dimension is the measurement index (the accumulation of Eq. (1),
// Sec. 2.1, in its particle-hole form).
//
// One measurement's operands are only 2 NQ N complex numbers (two diagonals of
// G per transfer), while G4 has NQ N^2 entries.  So the direct term is kept in
// operand form over a window of several batches and added to the single FP64
// accumulator acc[K1][K2][q][m] (which the exchange kernel updates every batch)
// once per window: one read-modify-write of G4 per window for this term.
//
//   k_pack_raw   every batch: a_r and b_r as complex64, measurement-fastest,
//                into the window: araw[Q][K][w], braw[Q][K][w] (w = window slot)
//   at the end of a window, for each group of up to kGroupQ transfers:
//   k_split      the group's operands as TF32 hi/lo planes (K-major, the
//                complex product embedded as real products, below)
//   k_direct_tc  the GEMM on the tensor cores into an FP32 scratch
//                [Ql][K1][K2] (plain coalesced stores); the tiles of Q = 0
//                accumulate each 32-element K chunk on its own and add the
//                partial sums to an FP64 scratch in a fixed order (for Q = 0 the
//                operands carry the coherent G0 part of every measurement in
//                the density channel or with a spin-split G0, and the tensor
//                cores' FP32 accumulation loses about one unit in the last place
//                of the running sum per MMA)
//   k_merge      acc[K1][K2][Q0 .. Q0+nQ) += scratch: one run of nQ entries per
//                (K1, K2), added by an asynchronous bulk FP64 reduction
//
// Real embedding of the complex GEMM (x ~ hi + lo in TF32 for every operand):
//   A [Ql][K2][kk]    = (Re b | Im b)            kk = w | Bw + w
//   B [Ql][0][K1][kk] = (Re a | -Im a)    ->  Re(b a) = A . B[0]
//   B [Ql][1][K1][kk] = (Im a |  Re a)    ->  Im(b a) = A . B[1]
// The GEMM computes Dir^T[K2][K1] so that the tensor-memory lanes (one thread
// each in the epilogue) run along K2: a warp's 32 lanes store 32 consecutive K2
// of one column K1 of the scratch, 256 contiguous bytes.  One output tile is 128
// rows K2 x 128 columns K1 of one transfer, [Re | Im] = 128 x 256 FP32 in tensor
// memory; per K step three MMAs (hi.hi + hi.lo + lo.hi) accumulate.
//
// Persistent GEMM kernel, one CTA per SM, warp roles:
//   warp 0      TMA producer (2-stage shared-memory ring, 96 KB per stage)
//   warp 1      MMA issuer (single thread), two TMEM accumulators (2 x 256 cols)
//   warps 2..9  epilogue
// Every mbarrier wait is bounded; on timeout the CTA records G4_DEV_TIMEOUT in
// the status word, stops issuing work, drains its own copies and returns.
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>
#include <new>

#include <type_traits>

#include "g4_gtilde.cuh"
#include "g4_internal.h"
#include "g4_ptx.cuh"

namespace {

using namespace g4ptx;

constexpr int kTileM = 128;          // rows K2 per tile
constexpr int kTileN = 128;          // complex columns K1 per tile (MMA N = 256)
constexpr int kRowBytes = 128;       // bytes of K per operand row and stage (swizzle span)
constexpr int kMmaPerStage = 4;      // MMAs per stage: 32 bytes of K each
// K elements per stage: 32 TF32 or 64 FP16 values
__host__ __device__ constexpr int kstage_of(bool f16) { return f16 ? 64 : 32; }
constexpr int kStages = 2;
constexpr int kAB = kTileM * kRowBytes;            // 16 KB: one A plane per stage
constexpr int kBB = 2 * kTileN * kRowBytes;        // 32 KB: one B plane per stage
constexpr int kStageBytes = 2 * kAB + 2 * kBB;     // 96 KB
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kTmemCols = 512;
// Epilogue run buffer per warp (tiles of Q = 0): 8 columns K1 x 32 lanes K2 of complex FP64.
constexpr int kRunCols = 8;
constexpr int kRunBytes = kRunCols * 32 * 16;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 256 + kEpiWarps * kRunBytes;
constexpr int kGroupQ = 16;          // transfers per flush group (scratch planes)
constexpr int kMergeK2 = 64;         // K2 per merge block

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ------------------------------------------------------------------ raw pack
// One block per (k, Q, 32-measurement chunk): a_r(K) and b_r(K) for K = (k, n),
// every n, through a shared tile so that the stores run along the window slot:
//   araw[Q][K][w0 + r] = a_r(K),  braw[Q][K][w0 + r] = b_r(K),  r < staged.
// a_r(K1) = 0 when K1 + Q leaves the frequency grid, b_r(K2) = 0 when K2 + Q does.
// The largest |component| of every a and b packed joins *wmax (FP32 bits), the
// window's maximum from which the FP16 split takes its scale.
__global__ void k_pack_raw(const float2* __restrict__ Gd, int staged, int w0, int Bw,
                           float2* __restrict__ araw, float2* __restrict__ braw,
                           const int* __restrict__ kadd, const int* __restrict__ ksub, G4Dims d,
                           unsigned* __restrict__ wmax) {
    __shared__ float2 ta[32][65];
    __shared__ float2 tb[32][65];
    const int k = blockIdx.x, Qi = blockIdx.y, r0 = blockIdx.z * 32;
    const int q = Qi / d.Nwex, m = d.m0 + Qi - q * d.Nwex;  // m: the transfer frequency
    const int Nw2 = d.Nw2, Nc = d.Nc;
    const size_t jstride = (size_t)Nc * d.ndn * Nc * Nw2;  // one (slot, spin)
    const int dkb = ksub[0 * Nc + q];                       // (-)q
    const int kq = kadd[k * Nc + q];
    const float ws = d.ch == G4_PH_DENSITY ? 1.f : -1.f;    // weight of spin -1
    float vmax = 0.f;
    for (int n0 = 0; n0 < Nw2; n0 += 64) {
        const int nw = min(64, Nw2 - n0);
        for (int t = threadIdx.x; t < 32 * 64; t += blockDim.x) {
            const int rr = t / 64, nn = t - rr * 64;
            const int r = r0 + rr, n = n0 + nn;
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
            if (r < staged && nn < nw && n + m < Nw2) {
                const float2* g0 = Gd + (size_t)(2 * r) * jstride;
                const float2* g1 = g0 + jstride;
                // a: G~(K1+Q, K1), diagonal (q, +m) at column K1 = (k, n)
                const size_t ia = (((size_t)q * d.ndn + (m + Nw2 - 1)) * Nc + k) * Nw2 + n;
                const float2 u0 = g0[ia], u1 = g1[ia];
                a = make_float2(u0.x + ws * u1.x, u0.y + ws * u1.y);
                // b: G~(K2, K2+Q), diagonal ((-)q, -m) at column K2+Q = (k (+) q, n + m)
                const size_t ib = (((size_t)dkb * d.ndn + (Nw2 - 1 - m)) * Nc + kq) * Nw2 + n + m;
                const float2 w0v = g0[ib], w1v = g1[ib];
                b = make_float2(w0v.x + ws * w1v.x, w0v.y + ws * w1v.y);
                vmax = fmaxf(vmax, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(b.x), fabsf(b.y))));
            }
            ta[rr][nn] = a;
            tb[rr][nn] = b;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 64 * 32; t += blockDim.x) {
            const int nn = t / 32, rr = t - nn * 32;
            const int r = r0 + rr;
            if (nn >= nw || r >= staged) continue;
            const size_t row = ((size_t)Qi * d.N + k * Nw2 + n0 + nn) * Bw + w0 + r;
            araw[row] = ta[rr][nn];
            braw[row] = tb[rr][nn];
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(wmax, __float_as_uint(vmax));
}

// ------------------------------------------------------------------ split
// Hi/lo planes of one transfer group for the first `fill` window slots (slots
// fill..Bwp-1 are written as zero), row stride Kst elements:
//   Ah/Al[Ql][K][w | Bwp + w] = (Re b | Im b)
//   Bh/Bl[Ql][0][K][...]      = (Re a | -Im a)
//   Bh/Bl[Ql][1][K][...]      = (Im a |  Re a)
// TF32 pairs x ~ hi + lo, or FP16 pairs x 2^s ~ hi + lo with the window's
// scale (f16_shift of *wmax).  One block per (K, Ql).
template <bool F16>
__device__ __forceinline__ void split_store(void* hp, void* lp, size_t i, float x, float scale) {
    if constexpr (F16) {
        const __half hi = __float2half_rn(x * scale);
        ((__half*)hp)[i] = hi;
        ((__half*)lp)[i] = __float2half_rn(x * scale - __half2float(hi));
    } else {
        const float hi = tf32_rna(x);
        ((float*)hp)[i] = hi;
        ((float*)lp)[i] = tf32_rna(x - hi);
    }
}

template <bool F16>
__global__ void k_split(const float2* __restrict__ araw, const float2* __restrict__ braw, int Q0,
                        int fill, int Bwp, int Bw, int Kst, void* __restrict__ Ah,
                        void* __restrict__ Al, void* __restrict__ Bh, void* __restrict__ Bl,
                        int N, const unsigned* __restrict__ wmax) {
    const int K = blockIdx.x, Ql = blockIdx.y;
    const float scale = F16 ? pow2f(f16_shift(*wmax)) : 1.f;
    const size_t src = ((size_t)(Q0 + Ql) * N + K) * Bw;
    const size_t ra = ((size_t)Ql * N + K) * Kst;
    const size_t rb0 = (((size_t)Ql * 2 + 0) * N + K) * Kst;
    const size_t rb1 = (((size_t)Ql * 2 + 1) * N + K) * Kst;
    for (int w = threadIdx.x; w < Bwp; w += blockDim.x) {
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (w < fill) {
            a = araw[src + w];
            b = braw[src + w];
        }
        split_store<F16>(Ah, Al, ra + w, b.x, scale);
        split_store<F16>(Ah, Al, ra + Bwp + w, b.y, scale);
        split_store<F16>(Bh, Bl, rb0 + w, a.x, scale);
        split_store<F16>(Bh, Bl, rb0 + Bwp + w, -a.y, scale);
        split_store<F16>(Bh, Bl, rb1 + w, a.y, scale);
        split_store<F16>(Bh, Bl, rb1 + Bwp + w, a.x, scale);
    }
}

// ------------------------------------------------------------------ GEMM
struct DParams {
    float2* scr;       // [nQ][N][N] FP32 results of the group (K1-major rows of K2)
    double2* scr0;     // [N][N] FP64 partial sums of Q = 0 (zeroed before the group)
    unsigned* status;
    int N, Nwex, Nw2, Q0;
    int Kw;            // K extent: 2 * padded window fill
    int nit, njt, ntiles;
    uint32_t idesc;
    const unsigned* wmax;  // FP16 operands: the window's largest |component| (FP32 bits)
    long long budget;  // clock64 cycles per wait
};


struct TileCoord {
    int Ql, i0, j0;
};

// Tile order: K1 tiles fastest, then K2 tiles, then the transfer, so that CTAs
// running at the same time share operand tiles in L2.
__device__ __forceinline__ TileCoord tile_coord(const DParams& P, int t) {
    const int jt = t % P.njt;
    t /= P.njt;
    const int it = t % P.nit;
    const int Ql = t / P.nit;
    return TileCoord{Ql, it * kTileM, jt * kTileN};
}

// Asynchronous FP64 reduction of a shared-memory run into global memory (the
// add is performed at L2), and the calling thread's bulk-group bookkeeping.
__device__ __forceinline__ void bulk_add_f64(double2* gdst, const double2* ssrc, uint32_t bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_u32(ssrc)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

template <bool F16>
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
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int nk = P.Kw / kstage_of(F16);  // stages of K per tile

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
                    const int kx = ks * kstage_of(F16);
                    tma_load_3d(st, &tmAh, &full[s], kx, tc.i0, tc.Ql);
                    tma_load_3d(st + kAB, &tmAl, &full[s], kx, tc.i0, tc.Ql);
                    tma_load_4d(st + 2 * kAB, &tmBh, &full[s], kx, tc.j0, 0, tc.Ql);
                    tma_load_4d(st + 2 * kAB + kBB / 2, &tmBh, &full[s], kx, tc.j0, 1, tc.Ql);
                    tma_load_4d(st + 2 * kAB + kBB, &tmBl, &full[s], kx, tc.j0, 0, tc.Ql);
                    tma_load_4d(st + 2 * kAB + kBB + kBB / 2, &tmBl, &full[s], kx, tc.j0, 1, tc.Ql);
                }
            }
            // after an abort, wait (bounded) until the copies already issued have landed
            if (*abort_flag) {
                for (uint32_t k = 0; k < (uint32_t)kStages && k < g; ++k) {
                    const uint32_t gg = g - 1 - k;
                    mbar_drain(&full[gg % kStages], (gg / kStages) & 1, kDrainBudget);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0, tl = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < P.ntiles && !*abort_flag; t += gridDim.x) {
                const bool split = P.Q0 + tile_coord(P, t).Ql == 0;
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
                    for (int k = 0; k < kMmaPerStage; ++k) {
                        const uint32_t off = k * 32;  // 8 TF32 or 16 FP16 = 32 bytes along K
                        const uint64_t ah = sdesc_k128(st + off), al = sdesc_k128(st + kAB + off);
                        const uint64_t bh = sdesc_k128(st + 2 * kAB + off);
                        const uint64_t bl = sdesc_k128(st + 2 * kAB + kBB + off);
                        const uint32_t acc0 = ((split ? 0 : ks) | k) != 0;
                        if constexpr (F16) {
                            mma_f16(d_tmem, ah, bh, P.idesc, acc0);
                            mma_f16(d_tmem, ah, bl, P.idesc, 1);
                            mma_f16(d_tmem, al, bh, P.idesc, 1);
                        } else {
                            mma_tf32(d_tmem, ah, bh, P.idesc, acc0);
                            mma_tf32(d_tmem, ah, bl, P.idesc, 1);
                            mma_tf32(d_tmem, al, bh, P.idesc, 1);
                        }
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
            mbar_drain(mdone, 0, kDrainBudget);
        }
    } else {
        // epilogue warps: lane quadrant from the warp index, column half from the warp group
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        double2* runbuf = (double2*)(smem + kStages * kStageBytes + 256) + (size_t)(warp - 2) * (kRunBytes / 16);
        // FP16 operands carry the window's scale 2^s each: products 2^(2s)
        const float unscale = F16 ? pow2f(-2 * f16_shift(*P.wmax)) : 1.f;
        uint32_t tl = 0;
        bool live = true;
        for (int t = blockIdx.x; live && t < P.ntiles; t += gridDim.x) {
            const TileCoord tc = tile_coord(P, t);
            const bool split = P.Q0 + tc.Ql == 0;
            const int nsub = split ? nk : 1;
            const int K2s = tc.i0 + quad * 32;
            const int nk2 = min(32, P.N - K2s);
            float2* srow = P.scr + (size_t)tc.Ql * P.N * P.N + K2s + lane;
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
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    const int c0 = half * 64 + c * 32;
                    float re[32], im[32];
                    tmem_ld32(tbase + c0, re);
                    tmem_ld32(tbase + kTileN + c0, im);
                    tmem_wait_ld();
#pragma unroll
                    for (int g = 0; g < 32; ++g) {
                        re[g] *= unscale;
                        im[g] *= unscale;
                    }
                    if (c == 1) {
                        // last read of the accumulator: hand it back to the MMA warp
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty[b]);
                    }
                    if (!split) {
                        // the warp's 32 K2 of one column K1: 256 contiguous bytes
                        if (lane < nk2) {
#pragma unroll
                            for (int g = 0; g < 32; ++g) {
                                const int K1 = tc.j0 + c0 + g;
                                if (K1 < P.N) srow[(size_t)K1 * P.N] = make_float2(re[g], im[g]);
                            }
                        }
                        continue;
                    }
                    // Q = 0: this K chunk's partial sums, staged in shared memory as
                    // FP64 runs of 32 K2 and added to the FP64 scratch one chunk after
                    // the other (every reduction completes before the next is issued)
#pragma unroll
                    for (int g = 0; g < 32; g += kRunCols) {
                        if (lane < kRunCols) bulk_wait_all();
                        __syncwarp();
#pragma unroll
                        for (int jj = 0; jj < kRunCols; ++jj)
                            runbuf[jj * 32 + lane] = make_double2((double)re[g + jj], f32_to_f64(im[g + jj]));
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane < kRunCols) {
                            const int K1 = tc.j0 + c0 + g + lane;
                            if (K1 < P.N && nk2 > 0)
                                bulk_add_f64(P.scr0 + (size_t)K1 * P.N + K2s, runbuf + lane * 32,
                                             (uint32_t)(16 * nk2));
                            bulk_commit();
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
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ------------------------------------------------------------------ merge
// acc[K1][K2][Q0 + ql] += scratch value of (ql, K1, K2) for ql < nQ, K2 in this
// block's range of kMergeK2; entries whose K1 + Q or K2 + Q leaves the frequency
// grid are structurally zero and add 0.  Each K2's run of nQ values (contiguous
// in the accumulator) is staged in shared memory as FP64 and added with one
// bulk reduction.  Grid (ceil(N / kMergeK2), N).
__global__ void __launch_bounds__(256) k_merge(const float2* __restrict__ scr,
                                               const double2* __restrict__ scr0,
                                               double2* __restrict__ acc, int Q0, int nQ, G4Dims d) {
    __shared__ __align__(16) double2 run[kMergeK2 * kGroupQ];
    const int K1 = blockIdx.y, K2b = blockIdx.x * kMergeK2;
    const int N = d.N;
    const int n1 = K1 % d.Nw2;
    const int cnt = nQ * kMergeK2;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int ql = t / kMergeK2, k2l = t - ql * kMergeK2;
        const int K2 = K2b + k2l;
        const int Q = Q0 + ql;
        const int m = d.m0 + Q % d.Nwex;   // the transfer frequency
        double2 v = make_double2(0.0, 0.0);
        if (K2 < N && n1 + m < d.Nw2 && K2 % d.Nw2 + m < d.Nw2) {
            if (Q == 0) {
                v = scr0[(size_t)K1 * N + K2];
            } else {
                const float2 f = scr[((size_t)ql * N + K1) * N + K2];
                v = make_double2(f32_to_f64(f.x), f32_to_f64(f.y));
            }
        }
        run[k2l * nQ + ql] = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < kMergeK2) {
        const int K2 = K2b + threadIdx.x;
        if (K2 < N)
            bulk_add_f64(acc + ((size_t)K1 * N + K2) * d.NQ + Q0, run + threadIdx.x * nQ,
                         (uint32_t)(16 * nQ));
        bulk_commit();
        bulk_wait_read_all();   // the shared run must outlive the reduction's read
    }
}

// The same addition into an accumulator of compensated FP32 pairs: one thread
// per entry, read, added and written back (no other writer while it runs).
__global__ void __launch_bounds__(256) k_merge_pair(const float2* __restrict__ scr,
                                                    const double2* __restrict__ scr0,
                                                    double2* __restrict__ acc, int Q0, int nQ,
                                                    G4Dims d) {
    const int K1 = blockIdx.y, K2b = blockIdx.x * kMergeK2;
    const int N = d.N;
    const int n1 = K1 % d.Nw2;
    for (int t = threadIdx.x; t < nQ * kMergeK2; t += blockDim.x) {
        const int ql = t % nQ, k2l = t / nQ;   // consecutive threads: consecutive entries
        const int K2 = K2b + k2l;
        const int Q = Q0 + ql;
        const int m = d.m0 + Q % d.Nwex;
        if (K2 >= N || n1 + m >= d.Nw2 || K2 % d.Nw2 + m >= d.Nw2) continue;
        float4* e4 = reinterpret_cast<float4*>(acc + ((size_t)K1 * N + K2) * d.NQ + Q);
        float4 a = *e4;
        if (Q == 0) {
            const double2 v = scr0[(size_t)K1 * N + K2];
            pair_add(a.x, a.z, v.x);
            pair_add(a.y, a.w, v.y);
        } else {
            const float2 f = scr[((size_t)ql * N + K1) * N + K2];
            pair_add(a.x, a.z, f.x);
            pair_add(a.y, a.w, f.y);
        }
        *e4 = a;
    }
}

// ------------------------------------------------------------------ host
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

struct DirectPlan {
    int Bw = 0;          // window capacity in measurements (multiple of 32)
    int fill = 0;        // measurements in the window
    int batches = 0;     // full batches the window holds
    int Kst = 0;         // row stride of the split planes (2 * Bw elements)
    int nQg = 0;         // transfers per group
    bool f16 = true;     // FP16 (else TF32) hi/lo planes
    float2* araw = nullptr;   // [NQ][N][Bw]
    float2* braw = nullptr;
    void *Ah = nullptr, *Al = nullptr, *Bh = nullptr, *Bl = nullptr;  // group planes
    unsigned* wmax = nullptr; // the window's largest |a|, |b| component (FP32 bits)
    float2* scr = nullptr;    // [nQg][N][N]
    double2* scr0 = nullptr;  // [N][N]
    CUtensorMap mAh, mAl, mBh, mBl;
};

bool encode_maps(const G4Dims& d, DirectPlan& X) {
    auto enc = get_encoder();
    if (!enc) return false;
    const cuuint64_t K = (cuuint64_t)X.Kst;
    const cuuint64_t eb = X.f16 ? 2 : 4;
    const CUtensorMapDataType dt = X.f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint32_t kst = (cuuint32_t)kstage_of(X.f16);
    const cuuint32_t es[4] = {1, 1, 1, 1};
    {
        const cuuint64_t dims[3] = {K, (cuuint64_t)d.N, (cuuint64_t)X.nQg};
        const cuuint64_t strides[2] = {K * eb, K * eb * d.N};
        const cuuint32_t box[3] = {kst, kTileM, 1};
        for (int i = 0; i < 2; ++i) {
            CUresult r = enc(i ? &X.mAl : &X.mAh, dt, 3,
                             i ? (void*)X.Al : (void*)X.Ah, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return false;
        }
    }
    {
        const cuuint64_t dims[4] = {K, (cuuint64_t)d.N, 2, (cuuint64_t)X.nQg};
        const cuuint64_t strides[3] = {K * eb, K * eb * d.N, K * eb * d.N * 2};
        const cuuint32_t box[4] = {kst, kTileN, 1, 1};
        for (int i = 0; i < 2; ++i) {
            CUresult r = enc(i ? &X.mBl : &X.mBh, dt, 4,
                             i ? (void*)X.Bl : (void*)X.Bh, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return false;
        }
    }
    return true;
}

template <typename T>
g4_status dalloc(g4_ctx* h, T** p, size_t count) {
    return g4_dalloc_bytes(h, (void**)p, count * sizeof(T));
}

}  // namespace

// The default window: as many full batches as fit in kWindowBudget bytes of
// raw operands, at most kMaxWindowBatches (the FP32 sums of the window's GEMM
// then run over at most 2 x 8 x 256 terms).
constexpr size_t kWindowBudget = (size_t)24 << 30;
constexpr int kMaxWindowBatches = 8;

g4_status direct_prepare(g4_ctx* h) {
    const G4Dims& d = h->d;
    DirectPlan* X = new (std::nothrow) DirectPlan();
    if (!X) return g4_fail(h, G4_ERR_OOM, "host allocation of the direct-term plan");
    h->dplan = X;
    const size_t per_meas = 2 * (size_t)d.NQ * d.N * sizeof(float2);
    int F = h->opt.direct_batches;
    if (F <= 0) {
        const size_t fit = kWindowBudget / std::max<size_t>(1, per_meas * (size_t)h->batch);
        F = (int)std::max<size_t>(1, std::min<size_t>(kMaxWindowBatches, fit));
    }
    X->batches = F;
    X->f16 = h->opt.operands == G4_OPERANDS_FP16;
    X->Bw = (F * h->batch + 31) / 32 * 32;   // 2 Bw: a whole number of 64-element stages
    X->Kst = 2 * X->Bw;
    X->nQg = std::min(kGroupQ, d.NQ);
    g4_status st;
    const size_t raw = (size_t)d.NQ * d.N * X->Bw;
    if ((st = dalloc(h, &X->araw, raw)) != G4_OK) return st;
    if ((st = dalloc(h, &X->braw, raw)) != G4_OK) return st;
    // operands whose frequency leaves the grid stay zero (the deferred pack
    // never writes them; the eager pack writes them as zero)
    cudaError_t ze = cudaMemset(X->araw, 0, raw * sizeof(float2));
    if (ze == cudaSuccess) ze = cudaMemset(X->braw, 0, raw * sizeof(float2));
    if (ze != cudaSuccess) return g4_cuda_fail(h, ze, "direct window clear");
    const size_t plane = (size_t)X->nQg * d.N * X->Kst * (X->f16 ? 2 : 4);   // bytes
    if ((st = dalloc(h, (char**)&X->Ah, plane)) != G4_OK) return st;
    if ((st = dalloc(h, (char**)&X->Al, plane)) != G4_OK) return st;
    if ((st = dalloc(h, (char**)&X->Bh, 2 * plane)) != G4_OK) return st;
    if ((st = dalloc(h, (char**)&X->Bl, 2 * plane)) != G4_OK) return st;
    if ((st = dalloc(h, &X->scr, (size_t)X->nQg * d.N * d.N)) != G4_OK) return st;
    if ((st = dalloc(h, &X->scr0, (size_t)d.N * d.N)) != G4_OK) return st;
    if ((st = dalloc(h, &X->wmax, 1)) != G4_OK) return st;
    cudaError_t e = cudaMemset(X->wmax, 0, sizeof(unsigned));
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "direct window maximum clear");
    if (!encode_maps(d, *X))
        return g4_fail(h, G4_ERR_CUDA, "cuTensorMapEncodeTiled failed for the direct-term operands");
    e = cudaFuncSetAttribute(X->f16 ? k_direct_tc<true> : k_direct_tc<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "direct smem attribute");
    return G4_OK;
}

void direct_window_ptrs(const g4_ctx* h, float2** araw, float2** braw, unsigned** wmax, int* fill,
                        int* Bw) {
    const DirectPlan* X = (const DirectPlan*)h->dplan;
    *araw = X ? X->araw : nullptr;  // no plan yet (the exchange tuner runs before it)
    *braw = X ? X->braw : nullptr;
    *wmax = X ? X->wmax : nullptr;
    *fill = X ? X->fill : 0;
    *Bw = X ? X->Bw : 0;
}

int direct_fill(const g4_ctx* h) {
    const DirectPlan* X = (const DirectPlan*)h->dplan;
    return X ? X->fill : 0;
}

int direct_window(const g4_ctx* h) {
    const DirectPlan* X = (const DirectPlan*)h->dplan;
    return X ? X->Bw : 0;
}

g4_status direct_pack(g4_ctx* h, int staged, bool* flush_due) {
    DirectPlan* X = (DirectPlan*)h->dplan;
    const G4Dims& d = h->d;
    if (X->fill + staged > X->Bw) return g4_fail(h, G4_ERR_STATE, "direct-term window overflow");
    // deferred staging: the exchange pack has already written the batch's
    // operands into the window (at the fill before this call)
    if (!h->deferred) {
        prof_begin(h, G4_K_PACK);
        k_pack_raw<<<dim3(d.Nc, d.NQ, (staged + 31) / 32), 256, 0, h->stream>>>(
            h->Gd, staged, X->fill, X->Bw, X->araw, X->braw, h->kadd, h->ksub, d, X->wmax);
        prof_end(h, G4_K_PACK);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return g4_cuda_fail(h, e, "direct pack launch");
    }
    X->fill += staged;
    *flush_due = X->fill + h->batch > X->Bw;
    return G4_OK;
}

g4_status direct_flush(g4_ctx* h) {
    DirectPlan* X = (DirectPlan*)h->dplan;
    if (!X || X->fill == 0) return G4_OK;
    const G4Dims& d = h->d;
    const int Bwp = (X->fill + 31) / 32 * 32;
    DParams P;
    P.scr = X->scr;
    P.scr0 = X->scr0;
    P.status = h->dstatus;
    P.N = d.N;
    P.Nwex = d.Nwex;
    P.Nw2 = d.Nw2;
    P.Kw = 2 * Bwp;
    P.nit = (d.N + kTileM - 1) / kTileM;
    P.njt = (d.N + kTileN - 1) / kTileN;
    P.idesc = X->f16 ? idesc_f16(kTileM, 2 * kTileN) : idesc_tf32(kTileM, 2 * kTileN);
    P.wmax = X->wmax;
    P.budget = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : 4000000000LL;
    cudaError_t e;
    for (int Q0 = 0; Q0 < d.NQ; Q0 += X->nQg) {
        const int nQ = std::min(X->nQg, d.NQ - Q0);
        if (Q0 == 0) {
            e = cudaMemsetAsync(X->scr0, 0, (size_t)d.N * d.N * sizeof(double2), h->stream);
            if (e != cudaSuccess) return g4_cuda_fail(h, e, "direct scratch clear");
        }
        prof_begin(h, G4_K_DIRECT_SPLIT);
        auto* split = X->f16 ? k_split<true> : k_split<false>;
        split<<<dim3(d.N, nQ), 256, 0, h->stream>>>(X->araw, X->braw, Q0, X->fill, Bwp, X->Bw,
                                                     X->Kst, X->Ah, X->Al, X->Bh, X->Bl, d.N, X->wmax);
        prof_end(h, G4_K_DIRECT_SPLIT);
        if ((e = cudaGetLastError()) != cudaSuccess) return g4_cuda_fail(h, e, "direct split launch");
        P.Q0 = Q0;
        P.ntiles = nQ * P.nit * P.njt;
        const int grid = P.ntiles < sm_count() ? P.ntiles : sm_count();
        prof_begin(h, G4_K_DIRECT);
        auto* gemm = X->f16 ? k_direct_tc<true> : k_direct_tc<false>;
        gemm<<<grid, kThreads, kSmemBytes, h->stream>>>(X->mAh, X->mAl, X->mBh, X->mBl, P);
        prof_end(h, G4_K_DIRECT);
        if ((e = cudaGetLastError()) != cudaSuccess) return g4_cuda_fail(h, e, "direct launch");
        prof_begin(h, G4_K_DIRECT_MERGE);
        auto* merge = h->opt.accum == G4_ACCUM_F32PAIR ? k_merge_pair : k_merge;
        merge<<<dim3((d.N + kMergeK2 - 1) / kMergeK2, d.N), 256, 0, h->stream>>>(
            X->scr, X->scr0, h->acc, Q0, nQ, d);
        prof_end(h, G4_K_DIRECT_MERGE);
        if ((e = cudaGetLastError()) != cudaSuccess) return g4_cuda_fail(h, e, "direct merge launch");
    }
    // the next window's maximum starts again
    if ((e = cudaMemsetAsync(X->wmax, 0, sizeof(unsigned), h->stream)) != cudaSuccess)
        return g4_cuda_fail(h, e, "direct window maximum clear");
    X->fill = 0;
    return G4_OK;
}

void direct_reset(g4_ctx* h) {
    DirectPlan* X = (DirectPlan*)h->dplan;
    if (!X) return;
    X->fill = 0;
    cudaMemsetAsync(X->wmax, 0, sizeof(unsigned), h->stream);
}

// The filled part of the window (both operand arrays, each [NQ][N][fill]
// complex64) to or from host memory, for checkpoints.  Synchronous.
g4_status direct_window_copy(g4_ctx* h, void* host, bool to_host) {
    DirectPlan* X = (DirectPlan*)h->dplan;
    if (!X || X->fill == 0) return G4_OK;
    const G4Dims& d = h->d;
    const size_t rows = (size_t)d.NQ * d.N, width = (size_t)X->fill * sizeof(float2);
    const size_t pitch = (size_t)X->Bw * sizeof(float2);
    char* hb = (char*)host;
    float2* dev[2] = {X->araw, X->braw};
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = to_host
            ? cudaMemcpy2D(hb + i * rows * width, width, dev[i], pitch, width, rows, cudaMemcpyDeviceToHost)
            : cudaMemcpy2D(dev[i], pitch, hb + i * rows * width, width, width, rows, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return g4_cuda_fail(h, e, "direct window copy");
    }
    return G4_OK;
}

size_t direct_window_bytes(const g4_ctx* h, int fill) {
    return 2 * (size_t)h->d.NQ * h->d.N * (size_t)fill * sizeof(float2);
}

// The window's largest operand component (FP32 bits) from / to the device,
// for checkpoints.  Synchronous.
g4_status direct_window_max(g4_ctx* h, unsigned* bits, bool to_host) {
    DirectPlan* X = (DirectPlan*)h->dplan;
    if (!X) {
        if (to_host) *bits = 0;
        return G4_OK;
    }
    cudaError_t e = to_host ? cudaMemcpy(bits, X->wmax, sizeof(unsigned), cudaMemcpyDeviceToHost)
                            : cudaMemcpy(X->wmax, bits, sizeof(unsigned), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? G4_OK : g4_cuda_fail(h, e, "direct window maximum copy");
}

g4_status direct_set_fill(g4_ctx* h, int fill) {
    DirectPlan* X = (DirectPlan*)h->dplan;
    if (!X) return fill == 0 ? G4_OK : g4_fail(h, G4_ERR_INVALID, "handle has no direct term");
    if (fill < 0 || fill > X->Bw) return g4_fail(h, G4_ERR_INVALID, "checkpoint window exceeds this handle's");
    X->fill = fill;
    return G4_OK;
}

void direct_release(g4_ctx* h) {
    DirectPlan* X = (DirectPlan*)h->dplan;
    if (!X) return;
    void* ptrs[] = {X->araw, X->braw, X->Ah, X->Al, X->Bh, X->Bl, X->scr, X->scr0, X->wmax};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete X;
    h->dplan = nullptr;
}
