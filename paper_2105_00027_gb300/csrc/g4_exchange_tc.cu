// Exchange-type term of the G4 update on the tcgen05 tensor cores.
//
// For a fixed difference D = K2 - K1 = (dk, dn) the exchange term of every
// channel is a product of two diagonals of the staged G~ = sqrt(s_r) G:
//
//   X_D(K1, P) = sum_j u_j(K1) w_j(P),        j = (measurement r, spin)
//   u_j(K1) = G~_j(K1+D, K1)                   (diagonal D, row K1)
//   w_j(P)  = G~_j'(P, P+D)  (ph channels: diagonal -D, row P+D; P = K1+Q)
//   w_j(P)  = G~_j'(P-D, P)  (pp channel:  diagonal -D, row P;   P = Q-K1)
//
// with j' = j (magnetic, density) or the opposite spin (transverse and the
// particle-particle form of Eq. (1), Sec. 2.1).  Only the band of columns P
// that differ from K1 by a transfer Q is wanted, so one output tile is
//   rows    (k1, n1) for kb momenta x nb frequencies of diagonal D,
//   columns (p, n') for pb momenta x a window of W = nb + Nwex - 1 frequencies
//           of diagonal -D, covering every transfer m of every row.
// The complex product is a real GEMM on interleaved (Re, Im) rows and columns:
// lanes 2i and 2i+1 of the accumulator hold the Re- and Im-rows of one K1, and
//   Re(u w) = C[Re][Re] - C[Im][Im],   Im(u w) = C[Re][Im] + C[Im][Re]
// are formed with one lane exchange in the epilogue.  The GEMM's K dimension
// is the batch of measurements times the two spins, so one tile accumulates a
// whole batch before it is added to the FP64 exchange accumulator
// acc[K1][K2][q][m] (the accumulation of Eq. (1), Sec. 2.1, batched).
//
// Precision: every operand is split x = hi + lo into two TF32 planes
// (k_pack_xtc) and each product is hi.hi + hi.lo + lo.hi with FP32
// accumulation, as for the direct term.  The tensor cores' FP32 accumulation
// loses about one unit in the last place of the running sum per MMA, and the
// diagonal D = 0 carries the coherent G0(K1) G0(P) part of every measurement
// (G0 is diagonal in K), so its sums grow linearly with the batch and that
// loss would reach 1e-6 relative at 64 measurements.  Tiles of D = 0 are
// therefore split along K inside their block: each 8-element K step gets its
// own accumulator whose three MMAs start from zero, and the epilogue adds every
// partial result to the FP64 accumulator in turn (one block owns all of them,
// so the read-modify-writes of one entry never overlap).
//
// Persistent kernel, one CTA per SM, warp roles:
//   warp 0      TMA producer: per 32-measurement chunk one stage of four 5-D
//               boxes (A hi/lo, B hi/lo), two stages
//   warp 1      MMA issuer (one thread), two tensor-memory accumulators
//   warps 2..17 epilogue (four per tensor-memory lane quarter, splitting the
//               column momenta): tensor-memory loads, complex combination,
//               FP64 runs staged in shared memory and added to the accumulator
//               by asynchronous bulk reductions
// Every mbarrier wait is bounded; on timeout the block records G4_DEV_TIMEOUT,
// stops issuing, drains its own copies and MMAs, frees its tensor memory and
// returns.
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <type_traits>

#include "g4_gtilde.cuh"
#include "g4_internal.h"
#include "g4_ptx.cuh"

namespace {

using namespace g4ptx;

constexpr int kEpiWarps = 16;
constexpr int kParts = kEpiWarps / 4;          // epilogue warps per tensor-memory lane quarter
constexpr int kRunBufs = 1;                    // FP64 run buffers per epilogue warp
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kStages = 2;
constexpr int kARows = 128;                    // MMA M
constexpr int kAPlane = kARows * 128;          // bytes of one A plane per stage
constexpr uint32_t kTmemCols = 512;            // two accumulators of up to 256 columns
constexpr int kMaxW = 16;                      // frequency window (columns per momentum / 2)
constexpr int kMaxNb = 8;                      // row frequencies per tile
constexpr int kRowBytes = 128;                 // bytes of one operand row per stage (swizzle span)
constexpr int kMmaPerStage = 4;                // MMAs per stage: 32 bytes of K each
// K (batch x spin) elements per stage: 32 TF32 or 64 FP16 values
__host__ __device__ constexpr int chunk_of(bool f16) { return f16 ? 64 : 32; }
constexpr int kSmemMax = 232448;               // opt-in shared memory per block (sm_100 family)

// Stride (in 16-byte entries) of the epilogue's FP64 runs in shared memory: at
// least Nwex and 2 mod 8, so that the 16-byte stores of the eight lanes of a
// quarter warp (four row pairs x Re/Im-lane) fall into distinct bank groups.
__host__ __device__ constexpr int run_stride(int Nwex) { return (Nwex + 5) / 8 * 8 + 2; }

__host__ __device__ constexpr int tc_smem_bytes(int N, int Nwex) {
    return kStages * (2 * (128 * 128) + 2 * N * 128) + 1024 + 256 +
           kEpiWarps * kRunBufs * 16 * run_stride(Nwex) * 16;
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ---------------------------------------------------------------- operand pack
// X[a][k][n][c][jj] for the diagonals D = dl[a] of one group: component c of
// G~_j((k (+) dk, n + dn), (k, n)), jj = spin * Jh + r, as a hi plane and a lo
// plane: TF32 values x ~ hi + lo, or FP16 values x 2^s ~ hi + lo with the
// batch's scale 2^s (f16_shift of the largest |G~| component, which the G
// build records in *gmax).  Only the rows on the grid (n + dn in [0, Nw2)) are
// written; the exchange kernel never uses the others.  Measurements r >=
// staged are zero.
//
// One block per (k, diagonal, 16 frequencies n): it stages every measurement
// and spin of its 16 rows in shared memory (reading 16 consecutive complex64
// of each slot, one 128-byte line), then writes each row's J values as one
// contiguous run per plane and component (16-byte vectors), so that every
// line of X is written whole by one block.
constexpr int kPackN = 16;

template <bool F16>
__global__ void __launch_bounds__(256) k_pack_xtc(const float2* __restrict__ Gd, int staged, int Jh,
                                                  const int2* __restrict__ dl,
                                                  void* __restrict__ Xh, void* __restrict__ Xl,
                                                  const unsigned* __restrict__ gmax, G4Dims d) {
    extern __shared__ float2 tile[];  // [2 Jh rows jj = spin * Jh + r][kPackN + 1]
    const int k = blockIdx.x, a = blockIdx.y;
    const int2 D = dl[a];
    const int dk = D.x, dn = D.y;
    const int Nw2 = d.Nw2, Nc = d.Nc, J = 2 * Jh;
    const int nlo = max(0, -dn), nhi = min(Nw2, Nw2 - dn);
    const int n0 = nlo + blockIdx.z * kPackN;
    const int nv = min(kPackN, nhi - n0);
    if (nv <= 0) return;
    const size_t jstride = (size_t)Nc * d.ndn * Nc * Nw2;
    const float2* src = Gd + (((size_t)dk * d.ndn + (dn + Nw2 - 1)) * Nc + k) * Nw2 + n0;
    const size_t rowbase = ((size_t)a * Nc + k) * Nw2 + n0;
    constexpr int ld = kPackN + 1;
    const float scale = F16 ? pow2f(f16_shift(*gmax)) : 1.f;
    constexpr int U = 8;  // loads in flight per thread
    const int nitem = J * kPackN;  // (jj, n)
    for (int t0 = threadIdx.x; t0 < nitem; t0 += U * blockDim.x) {
        float2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u * blockDim.x;
            v[u] = make_float2(0.f, 0.f);
            const int jj = t / kPackN, nn = t - jj * kPackN;
            const int sp = jj >= Jh ? 1 : 0, r = jj - sp * Jh;
            if (t < nitem && nn < nv && r < staged) v[u] = src[(size_t)(2 * r + sp) * jstride + nn];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t < nitem) tile[(t / kPackN) * ld + t % kPackN] = v[u];
        }
    }
    __syncthreads();
    // one thread writes the consecutive jj of one (n, c) that fill a 16-byte
    // vector (eight FP16 or four TF32 values) to each plane; lane pairs take
    // two neighbouring vectors of one row, so that every warp store writes
    // whole 32-byte sectors (16-byte pieces of 32 rows left half sectors that
    // L2 had to complete from DRAM), and the lanes of a half warp read eight
    // frequencies of two tile rows eight apart (conflict-free for FP16)
    constexpr int E = F16 ? 8 : 4;
    const int nseg = J / E;  // even: J is a multiple of 64
    for (int t = threadIdx.x; t < kPackN * 2 * nseg; t += blockDim.x) {
        const int rest = t >> 1;
        const int nn = rest % kPackN, c = (rest / kPackN) & 1, seg = (rest / (2 * kPackN)) * 2 + (t & 1);
        if (nn >= nv) continue;
        const size_t o = ((rowbase + nn) * 2 + c) * J + (size_t)seg * E;
        if constexpr (F16) {
            __align__(16) __half hi[8];
            __align__(16) __half lo[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float2 v = tile[(seg * 8 + u) * ld + nn];
                const float x = (c ? v.y : v.x) * scale;
                hi[u] = __float2half_rn(x);
                lo[u] = __float2half_rn(x - __half2float(hi[u]));
            }
            *reinterpret_cast<uint4*>((__half*)Xh + o) = *reinterpret_cast<const uint4*>(hi);
            *reinterpret_cast<uint4*>((__half*)Xl + o) = *reinterpret_cast<const uint4*>(lo);
        } else {
            float4 hi, lo;
            float* ph = &hi.x;
            float* pl = &lo.x;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 v = tile[(seg * 4 + u) * ld + nn];
                const float x = c ? v.y : v.x;
                ph[u] = tf32_round(x);
                pl[u] = tf32_round(x - ph[u]);
            }
            *reinterpret_cast<float4*>((float*)Xh + o) = hi;
            *reinterpret_cast<float4*>((float*)Xl + o) = lo;
        }
    }
}

// The direct term's window, when the deferred pack also writes its operands
// (channels with a direct term): a_r(K) into araw[Q][K][w0 + r], b_r(K) into
// braw[Q][K][w0 + r], the window holding Bw slots; ws = weight of spin -1;
// the largest |component| joins *wmax.
struct DirectOut {
    float2* araw;
    float2* braw;
    unsigned* wmax;
    int w0, Bw;
    float ws;
};

// Two FP32 values rounded to FP16 and packed into one register (a in the low
// half, b in the high half), and the halves back as FP32.
__device__ __forceinline__ uint32_t pack_f16x2(float a, float b) {
    uint32_t u;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(b), "f"(a));
    return u;
}
__device__ __forceinline__ float low_f16(uint32_t u) {
    return __half2float(__ushort_as_half((unsigned short)(u & 0xFFFFu)));
}
__device__ __forceinline__ float high_f16(uint32_t u) {
    return __half2float(__ushort_as_half((unsigned short)(u >> 16)));
}

template <bool F16, bool M64>
struct PackM {
    static constexpr int SL = F16 ? 32 : 16;          // slots per spin and tile
    static constexpr int EB = M64 ? 8 : 16;           // bytes of an entry of M
    static constexpr int ET = M64 ? 128 : 64;         // entries per tile
    static constexpr int THREADS = 512;
    static constexpr int QS = F16 ? 8 : 4;            // slots of a quarter (one 16-byte vector)
    static constexpr int QPAD = 32;                   // shift of each quarter group (bank spread)
    static constexpr int MBYTES = 2 * SL * ET * EB + (2 * SL / QS) * QPAD;  // M pieces of one stage
    // byte offset of (spin ss, slot us, entry e) in a stage: slot-major rows
    // of ET entries, every group of QS slots shifted by QPAD so that the four
    // quarters read by neighbouring lanes fall into different banks
    __host__ __device__ static constexpr int moff(int ss, int us, int e) {
        return ((ss * SL + us) * ET + e) * EB + ((ss * SL + us) / QS) * QPAD;
    }
    static constexpr int GBYTES = 2 * 2 * 128 * 8;    // shared G0: [spin][row kr | row k][2Nw <= 128] complex64
    static constexpr int STAGE = MBYTES + GBYTES;     // bytes of one stage
    static constexpr int NST = 3;                     // stages
    static constexpr int MAXNC = 256;
    // stages, D = 0 positions, slot sign factors, full and empty mbarriers, flag
    static constexpr int SMEM = NST * STAGE + MAXNC * 4 + kMaxBatch * 8 + 2 * NST * 8 + 16;
};

// Position of diagonal (dk, dn) in the exchange's diagonal list: (D, -D) pairs
// in the order dn = 0, 1, ... with dk inner, dn = 0 listed once per pair
// (pos0, a table of Nc entries); mk = (-)dk.
__device__ __forceinline__ int diag_pos(int dk, int dn, int mk, int Nc, const int* pos0) {
    if (dn > 0) return Nc + (dn - 1) * 2 * Nc + 2 * dk;
    if (dn < 0) return Nc + (-dn - 1) * 2 * Nc + 2 * mk + 1;
    return pos0[dk];
}

__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Deferred staging: the exchange operand planes (and, for channels with a
// direct term, the window's a and b) formed straight from the staged
// measurements' M, with no intermediate G.  The work is split into tiles: one
// (row momentum kr, column momentum k) block of M, ET entries of it (RI whole
// rows of 2Nw < ET columns, or ET columns of one row), and SL consecutive
// slots of both spins (SL = 32 FP16 or 16 TF32 values: a 64-byte half line of
// an X row per spin).  Persistent, one block per SM, each block a contiguous
// range of tiles (column momentum fastest).  A producer warp brings each
// tile's rows of M (one row piece per slot and spin) and, when every
// measurement shares one G0, the G0 of the tile's rows and columns into a ring
// of NST shared-memory stages with bulk copies that complete on the stage's
// full mbarrier, refilling a stage when its empty mbarrier says the 16
// consumer warps are done with it.  Consumers: four lanes per (entry, spin),
// each a quarter of the slots, form G~ from the staged M and write the half
// line of each plane and component of the row X[a(dk, dn)][k][n = j][c]
// (dk = kr (-) k, dn = i - j) as 16-byte vectors, the four lanes together one
// contiguous 64 bytes (whole sectors).  Then all consumer threads share the
// direct-term entries -- (dk, dn) = (q, m) for a(K1 = (k, j)), ((-)q, -m) for
// b(K2 = (kr, i)) -- writing both spins' weighted sum into the window.
// Entries whose diagonal lies outside the launch's group [a0, a0 + na) are
// skipped; slots r >= staged are zero in X and not written to the window.
// g0f: the G0 every staged measurement shares, as complex64 (its rows for the
// tile's two momenta arrive with the stage), or nullptr (each slot's own G0 is
// read).  FP16 pairs take their scale from *gscale (a largest |G~|
// component, FP32 bits); the largest component formed joins *gmax_out when it
// is given.  With redo != nullptr the launch does nothing unless *redo is set.
// Every mbarrier wait is bounded: on timeout the block records
// G4_DEV_TIMEOUT, waits (bounded) for the copies it issued and returns.  M and
// G0 must be 16-byte aligned (checked when a deferred handle stages a
// measurement).
template <bool F16, bool M64>
__global__ void __launch_bounds__(544, 1) k_pack_xtc_M(const __grid_constant__ G4SlotTable T, int staged,
                                                       int Jh, const float2* __restrict__ g0f,
                                                       const int* __restrict__ pos0g, int a0, int na,
                                                       void* __restrict__ Xh, void* __restrict__ Xl,
                                                       const unsigned* __restrict__ gscale,
                                                       unsigned* __restrict__ gmax_out,
                                                       const unsigned* __restrict__ redo, DirectOut D,
                                                       G4Dims d, long long budget,
                                                       unsigned* __restrict__ status) {
    if (redo && *redo == 0) return;
    using C = PackM<F16, M64>;
    using MV = typename std::conditional<M64, float2, double2>::type;
    constexpr int SL = C::SL, EB = C::EB, ET = C::ET, NST = C::NST;
    extern __shared__ __align__(128) unsigned char smem[];
    int* pos0 = reinterpret_cast<int*>(smem + NST * C::STAGE);
    float* srs = reinterpret_cast<float*>(pos0 + C::MAXNC);    // slot sign factors: magnitude
    int* sneg = reinterpret_cast<int*>(srs + kMaxBatch);         // and whether i times it
    uint64_t* bar = reinterpret_cast<uint64_t*>(sneg + kMaxBatch);  // full[NST], then empty[NST]
    uint64_t* ebar = bar + NST;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(ebar + NST);
    const int Nc = d.Nc, Nw2 = d.Nw2, N = d.N, Lx = d.Lx, Ly = d.Ly;
    const size_t NN = (size_t)N * N;
    // tile geometry: CJ columns of RI rows
    const int CJ = Nw2 < ET ? Nw2 : ET;
    const int ncb = (Nw2 + CJ - 1) / CJ;
    const int RI = Nw2 < ET ? ET / Nw2 : 1;
    const int ny = (Nw2 + RI - 1) / RI;
    const long long nkk = (long long)Nc * Nc;
    const long long ntiles = nkk * ny * ncb * (Jh / SL);
    const int tid = threadIdx.x;
    // consumer tasks: warp w takes entry groups G = w + 16 t (8 entries of one
    // spin: sp = G & 1, entries (G >> 1) * 8 + lane / 4), lane % 4 its quarter
    constexpr int QS = C::QS;
    constexpr int NTASK = ET * 2 * 4 / C::THREADS;
    const int qd = tid & 3;
    int te[NTASK], ti[NTASK], tj[NTASK], ts[NTASK];
#pragma unroll
    for (int tk = 0; tk < NTASK; ++tk) {
        const int G = (tid >> 5) + 16 * tk;
        ts[tk] = G & 1;
        te[tk] = (G >> 1) * 8 + ((tid & 31) >> 2);
        ti[tk] = te[tk] / CJ;
        tj[tk] = te[tk] - ti[tk] * CJ;
    }
    const float scale = F16 ? pow2f(f16_shift(*gscale)) : 1.f;
    const size_t J = 2 * (size_t)Jh;
    for (int t = tid; t < Nc; t += blockDim.x) pos0[t] = pos0g[t];
    for (int t = tid; t < staged; t += blockDim.x) {
        srs[t] = T.s[t].rs;
        sneg[t] = T.s[t].neg;
    }
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&bar[s], 1);
            mbar_init(&ebar[s], C::THREADS / 32);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // A block takes a contiguous range of tiles and walks it with counters
    // (column momentum fastest, then row momentum, column block, row block,
    // slot chunk); momenta are kept with their lattice components.
    struct Tile {
        int k, kr, kx, ky, krx, kry, cb, y, zc;
    };
    auto tile_at = [&](long long t) {
        Tile c;
        const int x = (int)(t % nkk);
        long long rest = t / nkk;
        c.kr = x / Nc;
        c.k = x - c.kr * Nc;
        c.kx = c.k % Lx;
        c.ky = c.k / Lx;
        c.krx = c.kr % Lx;
        c.kry = c.kr / Lx;
        c.cb = (int)(rest % ncb);
        rest /= ncb;
        c.y = (int)(rest % ny);
        c.zc = (int)(rest / ny);
        return c;
    };
    auto tile_next = [&](Tile& c) {
        if (++c.k < Nc) {
            if (++c.kx == Lx) {
                c.kx = 0;
                ++c.ky;
            }
            return;
        }
        c.k = c.kx = c.ky = 0;
        if (++c.kr < Nc) {
            if (++c.krx == Lx) {
                c.krx = 0;
                ++c.kry;
            }
            return;
        }
        c.kr = c.krx = c.kry = 0;
        if (++c.cb < ncb) return;
        c.cb = 0;
        if (++c.y < ny) return;
        c.y = 0;
        ++c.zc;
    };
    struct Geo {
        int kr, k, i0, ri, j0, cj, r0, dk, mk;
    };
    auto geo = [&](const Tile& c) {
        Geo g;
        g.kr = c.kr;
        g.k = c.k;
        g.i0 = c.y * RI;
        g.ri = min(RI, Nw2 - g.i0);
        g.j0 = c.cb * CJ;
        g.cj = min(CJ, Nw2 - g.j0);
        g.r0 = c.zc * SL;
        int dkx = c.krx - c.kx, dky = c.kry - c.ky;
        dkx += dkx < 0 ? Lx : 0;
        dky += dky < 0 ? Ly : 0;
        g.dk = dkx + Lx * dky;
        g.mk = (dkx ? Lx - dkx : 0) + Lx * (dky ? Ly - dky : 0);  // (-)dk
        return g;
    };
    const long long t_begin = (long long)blockIdx.x * ntiles / gridDim.x;
    const long long t_end = (long long)(blockIdx.x + 1) * ntiles / gridDim.x;
    // producer warp: the copies of tile c into stage s -- one row piece of M
    // per live slot, spin and row, and (shared G0) the complex64 G0 rows of the
    // tile's two momenta for both spins
    auto issue = [&](const Tile& c, int s) {
        const Geo g = geo(c);
        const int nlive = max(0, min(SL, staged - g.r0));
        const int ncopy = 2 * nlive * g.ri;
        const uint32_t piece = (uint32_t)g.cj * EB;
        unsigned char* st = smem + (size_t)s * C::STAGE;
        const uint32_t gbytes = g0f ? 4u * (uint32_t)Nw2 * 8u : 0u;
        if ((tid & 31) == 0) {
            const uint32_t bytes = (uint32_t)ncopy * piece + gbytes;
            if (bytes > 0) mbar_expect_tx(&bar[s], bytes);
            else mbar_arrive(&bar[s]);
        }
        __syncwarp();
        for (int c = tid & 31; c < ncopy; c += 32) {
            const int row = c % g.ri, rest = c / g.ri;
            const int us = rest % nlive, ss = rest / nlive;
            const unsigned char* src = reinterpret_cast<const unsigned char*>(T.s[g.r0 + us].M) +
                                       ((size_t)ss * NN + (size_t)(g.kr * Nw2 + g.i0 + row) * N +
                                        g.k * Nw2 + g.j0) * EB;
            bulk_load(st + C::moff(ss, us, row * CJ), src, piece, &bar[s]);
        }
        if (g0f && (tid & 31) < 4) {
            // [spin][0: row momentum kr | 1: column momentum k][2Nw] complex64
            const int z = (tid & 31) >> 1, col = (tid & 31) & 1;
            const float2* src = g0f + (size_t)z * N + (size_t)(col ? g.k : g.kr) * Nw2;
            bulk_load(st + C::MBYTES + (size_t)(z * 2 + col) * Nw2 * 8, src, (uint32_t)Nw2 * 8u, &bar[s]);
        }
    };
    float vmax = 0.f, dmax = 0.f;
    if (tid >= C::THREADS) {
        // producer warp: refill each stage once its consumer warps have released it
        int it = 0;
        Tile c = tile_at(t_begin);
        for (long long tt = t_begin; tt < t_end; ++tt, ++it, tile_next(c)) {
            const int s = it % NST;
            if (it >= NST && !mbar_wait(&ebar[s], (uint32_t)(it / NST - 1) & 1u, budget, abort_flag)) break;
            issue(c, s);
        }
        // no copy may be in flight when the block exits: wait (bounded) for
        // the last tiles issued (their copies have normally landed already)
        if ((tid & 31) == 0) {
            for (int k2 = 1; k2 <= NST && it - k2 >= 0; ++k2)
                mbar_drain(&bar[(it - k2) % NST], (uint32_t)((it - k2) / NST) & 1u, kDrainBudget);
            if (*abort_flag) atomicOr(status, (unsigned)G4_DEV_TIMEOUT);
        }
        return;
    }
    int it = 0;
    Tile tc = tile_at(t_begin);
    for (long long tt = t_begin; tt < t_end; ++tt, ++it, tile_next(tc)) {
        const int s = it % NST;
        const uint32_t ph = (uint32_t)(it / NST) & 1u;
        const Geo g = geo(tc);
        const int dk = g.dk, mk = g.mk;
        if (!mbar_wait(&bar[s], ph, budget, abort_flag)) {
            if ((tid & 31) == 0) atomicOr(status, (unsigned)G4_DEV_TIMEOUT);
            break;
        }
        const unsigned char* st = smem + (size_t)s * C::STAGE;
        const float2* sg0 = reinterpret_cast<const float2*>(st + C::MBYTES);  // [spin][kr | k][2Nw]
#pragma unroll
        for (int tk = 0; tk < NTASK; ++tk) {
            // task: 8 entries of one spin per warp, four lanes per entry, each
            // lane a quarter (QS slots, one 16-byte vector per plane and component)
            const int ee = te[tk], ii = ti[tk], jc = tj[tk], sp = ts[tk];
            if (!(ii < g.ri && jc < g.cj)) continue;
            const int i = g.i0 + ii, j = g.j0 + jc;
            const int a = diag_pos(dk, i - j, mk, Nc, pos0) - a0;
            if (a < 0 || a >= na) continue;
            const bool diag = g.kr == g.k && i == j;
            const size_t K1 = (size_t)g.kr * Nw2 + i, K2 = (size_t)g.k * Nw2 + j;
            float2 gi = make_float2(0.f, 0.f), gj = gi;
            if (g0f) {
                gi = sg0[(sp * 2 + 0) * Nw2 + i];
                gj = sg0[(sp * 2 + 1) * Nw2 + j];
            }
            const int u0 = qd * QS;              // the quarter's first slot in the tile
            const int rbase = g.r0 + u0;
            float ht[2][QS], lt[2][QS];
#pragma unroll
            for (int u = 0; u < QS; ++u) {
                const int r = rbase + u;
                float2 v = make_float2(0.f, 0.f);
                if (r < staged) {
                    if (!g0f) {
                        const double2 x1 = T.s[r].G0[sp * N + K1], x2 = T.s[r].G0[sp * N + K2];
                        gi = make_float2((float)x1.x, (float)x1.y);
                        gj = make_float2((float)x2.x, (float)x2.y);
                    }
                    // FP16: the power-of-two scale rides on the sign factor (the
                    // same bits as scaling afterwards); vmax is scaled too
                    const g4gt::SignFactor f{F16 ? srs[r] * scale : srs[r], sneg[r] != 0};
                    const MV m = *reinterpret_cast<const MV*>(st + C::moff(sp, u0 + u, ee));
                    v = g4gt::g_tilde(gi, g4gt::to_c64(m), gj, diag, f);
                    vmax = fmaxf(vmax, fmaxf(fabsf(v.x), fabsf(v.y)));
                }
                if constexpr (F16) {
                    ht[0][u] = v.x;
                    ht[1][u] = v.y;
                } else {
                    ht[0][u] = tf32_round(v.x);
                    ht[1][u] = tf32_round(v.y);
                    lt[0][u] = tf32_round(v.x - ht[0][u]);
                    lt[1][u] = tf32_round(v.y - ht[1][u]);
                }
            }
            const size_t o0 = ((((size_t)a * Nc + g.k) * Nw2 + j) * 2) * J + (size_t)sp * Jh + rbase;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const size_t o = o0 + (size_t)c * J;
                if constexpr (F16) {
                    uint32_t hq[QS / 2], lq[QS / 2];
#pragma unroll
                    for (int u2 = 0; u2 < QS / 2; ++u2) {
                        const float xa = ht[c][2 * u2], xb = ht[c][2 * u2 + 1];
                        hq[u2] = pack_f16x2(xa, xb);
                        lq[u2] = pack_f16x2(xa - low_f16(hq[u2]), xb - high_f16(hq[u2]));
                    }
                    *reinterpret_cast<uint4*>((__half*)Xh + o) = make_uint4(hq[0], hq[1], hq[2], hq[3]);
                    *reinterpret_cast<uint4*>((__half*)Xl + o) = make_uint4(lq[0], lq[1], lq[2], lq[3]);
                } else {
                    *reinterpret_cast<float4*>((float*)Xh + o) = make_float4(ht[c][0], ht[c][1], ht[c][2], ht[c][3]);
                    *reinterpret_cast<float4*>((float*)Xl + o) = make_float4(lt[c][0], lt[c][1], lt[c][2], lt[c][3]);
                }
            }
        }
        if (D.araw) {
            // the direct term's operands, spread over all threads: item = (row,
            // kind a or b, slot, transfer m), m fastest (neighbouring entries of
            // a row, then slots: few shared-memory bank conflicts); a at dn = m
            // (momentum difference q = dk), b at dn = -m (q = (-)dk); both
            // spins' weighted sum of the entry into the window
            const int nitem = g.ri * 2 * d.Nwex * SL;
            for (int t = tid; t < nitem; t += C::THREADS) {
                const int ml = t % d.Nwex;
                int rest = t / d.Nwex;
                const int us = rest % SL;
                rest /= SL;
                const int kind = rest & 1, ri2 = rest >> 1;
                const int r = g.r0 + us;
                const int q = kind ? mk : dk;
                if (r >= staged || q >= d.Nkex) continue;
                const int dnn = kind ? -(d.m0 + ml) : d.m0 + ml;
                const int ia = g.i0 + ri2, ja = ia - dnn;
                if (ja < g.j0 || ja >= g.j0 + g.cj) continue;
                const int ad = diag_pos(dk, dnn, mk, Nc, pos0) - a0;
                if (ad < 0 || ad >= na) continue;
                const int ea = ri2 * CJ + (ja - g.j0);
                const size_t k1 = (size_t)g.kr * Nw2 + ia, k2 = (size_t)g.k * Nw2 + ja;
                const bool dg = g.kr == g.k && ia == ja;
                const g4gt::SignFactor f{srs[r], sneg[r] != 0};
                float2 w = make_float2(0.f, 0.f);
#pragma unroll
                for (int z = 0; z < 2; ++z) {
                    float2 y1, y2;
                    if (g0f) {
                        y1 = sg0[(z * 2 + 0) * Nw2 + ia];
                        y2 = sg0[(z * 2 + 1) * Nw2 + ja];
                    } else {
                        const double2 x1 = T.s[r].G0[z * N + k1], x2 = T.s[r].G0[z * N + k2];
                        y1 = make_float2((float)x1.x, (float)x1.y);
                        y2 = make_float2((float)x2.x, (float)x2.y);
                    }
                    const MV m = *reinterpret_cast<const MV*>(st + C::moff(z, us, ea));
                    const float2 v = g4gt::g_tilde(y1, g4gt::to_c64(m), y2, dg, f);
                    w = z ? make_float2(w.x + D.ws * v.x, w.y + D.ws * v.y) : v;
                }
                dmax = fmaxf(dmax, fmaxf(fabsf(w.x), fabsf(w.y)));
                const size_t row = (size_t)(q * d.Nwex + ml) * N + (kind ? k1 : k2);
                (kind ? D.braw : D.araw)[row * D.Bw + D.w0 + r] = w;
            }
        }
        // the stage is read: release it to the producer
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&ebar[s]);
    }
    if (*abort_flag) return;  // the producer waits for its copies
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    }
    if ((tid & 31) == 0) {
        if (gmax_out) atomicMax(gmax_out, __float_as_uint(F16 ? vmax / scale : vmax));  // exact: 2^k
        if (D.araw) atomicMax(D.wmax, __float_as_uint(dmax));
    }
}

// The G0 every staged measurement shares, as the complex64 values the G~
// routine takes (rounded as the G build rounds them), for the deferred pack.
__global__ void k_g0_narrow(const double2* __restrict__ in, float2* __restrict__ out, int n) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        out[t] = make_float2((float)in[t].x, (float)in[t].y);
}

// The FP16 operand scale of a deferred handle, kept from batch to batch while
// it stays good: after a pack formed with the scale of *gscale, compare the
// shifts of the batch's largest component (*gmax) and of *gscale; if they
// differ by more than one (the largest scaled value would leave
// [2^12, 2^15): FP16 overflow, or more than one bit of the pairs' range
// unused) or no scale is set yet, take the batch's own and set *redo, so that
// the pack runs again with it.
__global__ void k_scale_check(const unsigned* __restrict__ gmax, unsigned* __restrict__ gscale,
                              unsigned* __restrict__ redo) {
    if (threadIdx.x != 0) return;
    const unsigned g = *gmax, s = *gscale;
    const int ds = f16_shift(s) - f16_shift(g);
    if (s == 0u || ds > 1 || ds < -1) {
        *gscale = g;
        *redo = 1u;
    } else {
        *redo = 0u;
    }
}

// ---------------------------------------------------------------- tensor-core kernel
struct TParams {
    double2* acc;
    unsigned* status;
    const int4* work;      // per (D, row-frequency block):
                           // {aD | bD << 16, dk, dn, n0 | split << 10}
    int Lx, Ly;            // cluster shape, k = kx + Lx ky
    uint32_t mLx;          // ceil(2^24 / Lx): k / Lx = (k mLx) >> 24 for k < 2^16
    int Nc, Nw2, N, Nwex, Nkex, NQ;
    int m0;                // first transfer frequency of the handle's slab
    int kb, nb, W, pb, nkb, npb;
    int nchunk, aoff;      // K chunks per tile; chunk offset of A (opposite spin)
    int ntiles;
    int run;               // consecutive tiles a block takes before the next block's turn
    int bplane;            // bytes of one B plane per stage (MMA N x 128)
    uint32_t txbytes;      // bytes the four boxes of a stage deliver
    uint32_t idesc;
    const unsigned* gmax;  // FP16 operands: largest |G~| component of the batch (FP32 bits)
    int pair;              // accumulator of compensated FP32 pairs (else FP64)
    long long budget;
};

struct XTile {
    int aD, bD, dk, dn, n0, kblk, pblk;
    int split;             // 1: one accumulator per K step (diagonal D = 0)
};

__device__ __forceinline__ XTile decode(const TParams& P, int t) {
    const int per = P.nkb * P.npb;
    const int e = t / per, r = t - e * per;
    const int4 w = P.work[e];
    XTile x;
    x.aD = w.x & 0xFFFF;
    x.bD = (int)((unsigned)w.x >> 16);
    x.dk = w.y;
    x.dn = w.z;
    x.n0 = w.w & 1023;
    x.split = (w.w >> 10) & 1;
    x.kblk = r / P.npb;
    x.pblk = r - x.kblk * P.npb;
    return x;
}

// The i-th tile of this block: runs of P.run consecutive tiles (which share
// operand rows) dealt round-robin to the blocks.  Increasing in i.
__device__ __forceinline__ int tile_of(const TParams& P, int i) {
    return ((i / P.run) * (int)gridDim.x + (int)blockIdx.x) * P.run + i % P.run;
}

// Lattice momenta k = kx + Lx ky, added componentwise modulo (Lx, Ly); the
// division by Lx uses a 24-bit reciprocal, exact for k < 2^16.
__device__ __forceinline__ void k_split(const TParams& P, int k, int& kx, int& ky) {
    ky = (int)(((uint64_t)(uint32_t)k * P.mLx) >> 24);
    kx = k - ky * P.Lx;
}

// Accumulator row of this thread's K1 in a tile (with K2 = K1 + D).
struct XRow {
    int k1, n1, n2;
    int k1x, k1y, k2x, k2y;
    bool ok;
    double2* base;         // &acc[K1][K2][0][0]
};

__device__ __forceinline__ XRow row_of(const TParams& P, const XTile& x, int i, int k_l, int n_l) {
    XRow r;
    r.k1 = x.kblk * P.kb + k_l;
    r.n1 = x.n0 + n_l;
    r.n2 = r.n1 + x.dn;
    r.ok = i < P.kb * P.nb && r.k1 < P.Nc && r.n1 < P.Nw2 && r.n2 >= 0 && r.n2 < P.Nw2;
    int dkx, dky;
    k_split(P, r.ok ? r.k1 : 0, r.k1x, r.k1y);
    k_split(P, x.dk, dkx, dky);
    r.k2x = r.k1x + dkx;
    r.k2y = r.k1y + dky;
    if (r.k2x >= P.Lx) r.k2x -= P.Lx;
    if (r.k2y >= P.Ly) r.k2y -= P.Ly;
    const int k2 = r.k2x + P.Lx * r.k2y;
    r.base = P.acc + ((size_t)(r.k1 * P.Nw2 + r.n1) * P.N + (size_t)(k2 * P.Nw2 + r.n2)) * P.NQ;
    return r;
}

// Transfer momentum q of output column momentum kp for this row (P.Nkex when
// the column holds no wanted transfer): particle-hole q = (kp (-) dk) (-) k1 =
// kp (-) k2, particle-particle q = kp (+) k1.
template <int V>
__device__ __forceinline__ int q_of(const TParams& P, const XRow& r, int kp) {
    if (!r.ok || kp >= P.Nc) return P.Nkex;
    int qx, qy;
    k_split(P, kp, qx, qy);
    if (V == 0) {
        qx -= r.k2x;
        qy -= r.k2y;
        if (qx < 0) qx += P.Lx;
        if (qy < 0) qy += P.Ly;
    } else {
        qx += r.k1x;
        qy += r.k1y;
        if (qx >= P.Lx) qx -= P.Lx;
        if (qy >= P.Ly) qy -= P.Ly;
    }
    return qx + P.Lx * qy;
}

// Complex results of one column momentum for this thread's row: tensor-memory
// load of its 2W columns, Re/Im combination across the lane pair, shift of the
// window so that transfer m = 0 comes first, and a second exchange after which
// lane c holds m = 2u + c as (Re, Im).  Warp-collective.
template <int NWH, int WM>
__device__ __forceinline__ void combine(uint32_t taddr, int nx8, int c, int shift, float unscale,
                                        float2 (&val)[NWH]) {
    float v[2 * WM];
#pragma unroll
    for (int u = 0; u < 2 * WM; ++u) v[u] = 0.f;
    tmem_ld8(taddr, v);
#pragma unroll
    for (int u = 1; u < WM / 4; ++u)
        if (u < nx8) tmem_ld8(taddr + 8 * u, v + 8 * u);
    tmem_wait_ld();
    float res[WM];
#pragma unroll
    for (int n = 0; n < WM; ++n) {
        const float y = __shfl_xor_sync(0xffffffffu, v[2 * n + 1], 1);
        res[n] = (c ? v[2 * n] + y : v[2 * n] - y) * unscale;
    }
    if (shift & 1) {
#pragma unroll
        for (int n = 0; n + 1 < WM; ++n) res[n] = res[n + 1];
    }
    if (shift & 2) {
#pragma unroll
        for (int n = 0; n + 2 < WM; ++n) res[n] = res[n + 2];
    }
    if (shift & 4) {
#pragma unroll
        for (int n = 0; n + 4 < WM; ++n) res[n] = res[n + 4];
    }
#pragma unroll
    for (int u = 0; u < NWH; ++u) {
        const float y = __shfl_xor_sync(0xffffffffu, c ? res[2 * u] : res[2 * u + 1], 1);
        val[u] = c ? make_float2(y, res[2 * u + 1]) : make_float2(res[2 * u], y);
    }
}

// Asynchronous reduction of a run of FP64 values from shared memory into
// global memory (the add is performed at L2): bytes is a multiple of 16, both
// addresses 16-byte aligned.  bulk_commit closes the thread's current group
// (an empty one if nothing was issued).
__device__ __forceinline__ void bulk_add_f64(double2* gdst, const double2* ssrc, uint32_t bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_u32(ssrc)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// V = 0: particle-hole geometry (w at P + D, P = K1 + Q, subtract);
// V = 1: particle-particle geometry (w at P, P = Q - K1, add).
// NWH: transfers per lane in the epilogue (Nwex <= 2 NWH); WM: bound of the
// frequency window W (register arrays of the epilogue).
template <int V, int NWH, int WM, bool F16>
__global__ void __launch_bounds__(kThreads, 1)
    k_exchange_tc(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                  const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                  TParams P) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int stage_bytes = 2 * kAPlane + 2 * P.bplane;
    uint64_t* bars = (uint64_t*)(smem + kStages * stage_bytes);
    uint64_t* full = bars;                 // [kStages]
    uint64_t* empty = bars + kStages;      // [kStages]
    uint64_t* tfull = bars + 2 * kStages;  // [2]
    uint64_t* tempty = tfull + 2;          // [2]
    uint64_t* mdone = tempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(mdone + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // Rows of a stage that no box writes (MMA rows beyond the A box, columns
    // beyond the B box) only feed accumulator entries the epilogue ignores;
    // clear them once so that they hold finite values.
    for (int i = threadIdx.x; i < kStages * stage_bytes / 16; i += blockDim.x)
        ((uint4*)smem)[i] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;
            for (int it = 0; !*abort_flag; ++it) {
                const int t = tile_of(P, it);
                if (t >= P.ntiles) break;
                const XTile x = decode(P, t);
                const int ak = x.kblk * P.kb;
                const int bn = (V == 0 ? x.n0 + x.dn : P.Nw2 - x.n0 - P.nb) + P.m0;
                const int bk = x.pblk * P.pb;
                bool ok = true;
                for (int ch = 0; ch < P.nchunk; ++ch, ++g) {
                    const int s = g % kStages;
                    const uint32_t ph = (g / kStages) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1, P.budget, abort_flag)) {
                        ok = false;
                        break;
                    }
                    uint8_t* st = smem + s * stage_bytes;
                    mbar_expect_tx(&full[s], P.txbytes);
                    int ca = ch + P.aoff;
                    if (ca >= P.nchunk) ca -= P.nchunk;
                    const int ja = ca * chunk_of(F16), jb = ch * chunk_of(F16);
                    tma_load_5d(st, &tmAh, &full[s], ja, 0, x.n0, ak, x.aD);
                    tma_load_5d(st + kAPlane, &tmAl, &full[s], ja, 0, x.n0, ak, x.aD);
                    tma_load_5d(st + 2 * kAPlane, &tmBh, &full[s], jb, 0, bn, bk, x.bD);
                    tma_load_5d(st + 2 * kAPlane + P.bplane, &tmBl, &full[s], jb, 0, bn, bk, x.bD);
                }
                if (!ok) break;
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
            for (int it = 0; ok && !*abort_flag; ++it) {
                const int t = tile_of(P, it);
                if (t >= P.ntiles) break;
                const bool split = decode(P, t).split != 0;
                uint32_t d_tmem = 0;
                if (!split) {
                    const int b = tl & 1;
                    if (!mbar_wait(&tempty[b], ((tl >> 1) & 1) ^ 1, P.budget, abort_flag)) break;
                    tc_fence_after();
                    d_tmem = tmem_base + (uint32_t)(b * 256);
                }
                for (int ch = 0; ch < P.nchunk; ++ch, ++g) {
                    const int s = g % kStages;
                    const uint32_t ph = (g / kStages) & 1;
                    if (!mbar_wait(&full[s], ph, P.budget, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + s * stage_bytes);
                    for (int k = 0; k < kMmaPerStage; ++k) {
                        if (split) {
                            const int b = tl & 1;
                            if (!mbar_wait(&tempty[b], ((tl >> 1) & 1) ^ 1, P.budget, abort_flag)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            d_tmem = tmem_base + (uint32_t)(b * 256);
                        }
                        const uint32_t off = k * 32;  // 8 TF32 or 16 FP16 = 32 bytes along K
                        const uint64_t ah = sdesc_k128(st + off);
                        const uint64_t al = sdesc_k128(st + kAPlane + off);
                        const uint64_t bh = sdesc_k128(st + 2 * kAPlane + off);
                        const uint64_t bl = sdesc_k128(st + 2 * kAPlane + P.bplane + off);
                        const uint32_t acc0 = (split || (ch | k) == 0) ? 0u : 1u;
                        if constexpr (F16) {
                            mma_f16(d_tmem, ah, bh, P.idesc, acc0);
                            mma_f16(d_tmem, ah, bl, P.idesc, 1);
                            mma_f16(d_tmem, al, bh, P.idesc, 1);
                        } else {
                            mma_tf32(d_tmem, ah, bh, P.idesc, acc0);
                            mma_tf32(d_tmem, ah, bl, P.idesc, 1);
                            mma_tf32(d_tmem, al, bh, P.idesc, 1);
                        }
                        if (split) {
                            mma_commit(&tfull[tl & 1]);
                            ++tl;
                        }
                    }
                    if (!ok) break;
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                if (!split) {
                    mma_commit(&tfull[tl & 1]);
                    ++tl;
                }
            }
            // wait (bounded) for every MMA this thread issued before tensor memory is freed
            mma_commit(mdone);
            mbar_drain(mdone, 0, kDrainBudget);
        }
    } else {
        // Epilogue: per column momentum, the lane pair of a row forms the complex
        // results of its window (combine), writes them as the FP64 run
        // acc[K1][K2][q][0..Nwex) into the warp's run buffer in shared memory, and
        // the pair's first lane adds the run to the accumulator with one
        // asynchronous bulk reduction (performed at L2, so no load round trip
        // holds up the epilogue).  Two run buffers per warp alternate; before a
        // buffer is rewritten its reductions must have read it.  The partial
        // sums of a split tile (D = 0) go to the same entries, so there every
        // reduction completes before the next one is issued (a fixed order of
        // additions).
        const int ew = warp - 2;
        // FP16 operands carry the batch's scale 2^s each: products 2^(2s)
        const float unscale = F16 ? pow2f(-2 * f16_shift(*P.gmax)) : 1.f;
        const int quad = warp & 3;             // tensor-memory lane quarter of this warp
        const int part = ew >> 2;              // column momenta kp_l = part, part + kParts, ...
        const int row = quad * 32 + lane;
        const int c = row & 1, i = row >> 1;   // Re/Im row, K1 index within the tile
        const int n_l = i % P.nb, k_l = i / P.nb;
        const int shift = V == 0 ? n_l : P.nb - 1 - n_l;  // window column of m = 0
        const int nx8 = (2 * P.W + 7) / 8;
        const int rs = run_stride(P.Nwex);
        double2* runs = (double2*)(smem + kStages * stage_bytes + 256) + (size_t)ew * kRunBufs * 16 * rs;
        const int pr = lane >> 1;              // row pair of this lane within the warp
        uint32_t tl = 0, wb = 0;
        bool live = true;
        for (int it = 0; live; ++it) {
            const int t = tile_of(P, it);
            if (t >= P.ntiles) break;
            const XTile x = decode(P, t);
            const XRow rw = row_of(P, x, i, k_l, n_l);
            // transfers m0 + m, m < mlim, of this row exist on the grid
            const int mlim = !rw.ok ? 0
                             : max(0, V == 0 ? min(P.Nwex, min(P.Nw2 - rw.n1, P.Nw2 - rw.n2) - P.m0)
                                             : min(P.Nwex, min(rw.n1, rw.n2) + 1 - P.m0));
            const int nsub = x.split ? P.nchunk * kMmaPerStage : 1;
            for (int sub = 0; sub < nsub; ++sub, ++tl) {
                const int b = tl & 1;
                const uint32_t tph = (tl >> 1) & 1;
                if (!mbar_wait(&tfull[b], tph, P.budget, abort_flag)) {
                    live = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * 256);
                // Column momenta of this warp: kp = part*step + j*kParts*step + h, h < step.
                // With step 2 the two results of a row for kp and kp+1 go to one buffer:
                // when their transfers are consecutive (q1 = q0 + 1, the usual case: the
                // column momenta of a tile run along the lattice's x direction, so do
                // q = kp (-) k2 up to one wrap) the 2 Nwex entries are one contiguous run of
                // the accumulator and one reduction adds them, half as many as one per kp.
                // Split tiles keep one kp per pass (their reductions complete one by one).
                const int step = (!x.split && !P.pair && 2 * P.Nwex <= rs) ? 2 : 1;
                if (part * step >= P.pb) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tempty[b]);
                }
                for (int k0 = part * step; k0 < P.pb; k0 += kParts * step) {
                    double2* buf = runs + ((size_t)wb * 16 + pr) * rs;
                    int qv[2] = {P.Nkex, P.Nkex};
                    const int nh = min(step, P.pb - k0);
                    for (int h = 0; h < nh; ++h) {
                        const int kp_l = k0 + h;
                        float2 val[NWH];
                        combine<NWH, WM>(tb + (uint32_t)(2 * P.W * kp_l), nx8, c, shift, unscale, val);
                        if (h == nh - 1 && k0 + kParts * step >= P.pb) {
                            // this warp's last read of the accumulator: hand it back to the MMA warp
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&tempty[b]);
                        }
                        qv[h] = q_of<V>(P, rw, x.pblk * P.pb + kp_l);
                        if (P.pair) {
                            // compensated FP32 pairs: this lane's transfers m = 2u + c of
                            // the row, read, added and written back (each entry has one
                            // writer per batch; a split tile's partial sums come from
                            // the same lane, in order)
                            if (mlim > 0 && qv[h] < P.Nkex) {
                                float4* e4 = reinterpret_cast<float4*>(rw.base + (size_t)qv[h] * P.Nwex);
#pragma unroll
                                for (int u = 0; u < NWH; ++u) {
                                    const int m = 2 * u + c;
                                    if (m < mlim)
                                        pair_add_c(e4 + m, V == 0 ? -val[u].x : val[u].x,
                                                   V == 0 ? -val[u].y : val[u].y);
                                }
                            }
                            continue;
                        }
                        if (h == 0) {
                            // the reductions that read this buffer (kRunBufs passes ago) are done reading
                            if (c == 0) {
                                if (x.split) bulk_wait_all();
                                else bulk_wait_read<kRunBufs - 1>();
                            }
                            __syncwarp();
                        }
#pragma unroll
                        for (int u = 0; u < NWH; ++u) {
                            const int m = 2 * u + c;
                            if (m < P.Nwex)
                                buf[h * P.Nwex + m] =
                                    m < mlim ? make_double2((double)(V == 0 ? -val[u].x : val[u].x), f32_to_f64(val[u].y, V == 0))
                                             : make_double2(0.0, 0.0);
                        }
                    }
                    if (P.pair) continue;
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (c == 0) {
                        if (mlim > 0) {
                            if (nh == 2 && qv[1] < P.Nkex && qv[1] == qv[0] + 1) {
                                // both transfers' full runs (entries m >= mlim are structurally
                                // zero and receive an exact zero)
                                bulk_add_f64(rw.base + (size_t)qv[0] * P.Nwex, buf, (uint32_t)(32 * P.Nwex));
                            } else {
                                // only the transfers on the grid: the entries with m >= mlim
                                // are structurally zero and never touched
                                for (int h = 0; h < nh; ++h)
                                    if (qv[h] < P.Nkex)
                                        bulk_add_f64(rw.base + (size_t)qv[h] * P.Nwex, buf + h * P.Nwex,
                                                     (uint32_t)(16 * mlim));
                            }
                        }
                        bulk_commit();  // one group per pass, so that "all but the last" is the other buffer
                    }
                    wb = wb + 1 == kRunBufs ? 0 : wb + 1;
                }
            }
        }
        if (c == 0) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) atomicOr(P.status, (unsigned)G4_DEV_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ---------------------------------------------------------------- host plan
struct XtcPlan {
    int kb = 0, nb = 0, W = 0, pb = 0, nkb = 0, npb = 0, N = 0;
    std::vector<int2> dl;                       // diagonals, in (D, -D) pairs
    std::vector<int> itemlen;                   // 2 for a pair, 1 for D = -D
    size_t work_bytes = 0;
    int Jh = 0, J = 0, aoff = 0;
    int gcap = 0;                               // diagonals per group (X slots)
    std::vector<int> gw0, gwn, gd0, gdn;        // per group: work entries, diagonals
    std::vector<int> gs0, gsn;                  // per group: split work entries (D = 0)
    int4* work = nullptr;
    int2* dlist = nullptr;
    int* pos0 = nullptr;                        // [Nc]: position of (dk, 0) in dl
    int packm_grid = 0;                         // blocks of the persistent pack from M
    float2* g0f = nullptr;                      // [2][N]: the shared G0 as complex64 (deferred)
    bool f16 = true;                            // FP16 (else TF32) hi/lo operand planes
    void* Xh = nullptr;
    void* Xl = nullptr;
    size_t xbytes = 0;
    size_t held = 0;                            // device bytes this plan allocated
    CUtensorMap mAh, mAl, mBh, mBl;
    int smem = 0, pack_smem = 0;
};

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
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

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

// Tile shapes that fit the MMA (2 kb nb <= 128 rows, N = 2 W pb <= 256
// columns rounded up to 16) and shared memory, ordered by a cost model: per
// row frequency, the larger of a tile's MMA work (~N) and its operand traffic
// (~(128 + N) x 2/3, equal to the MMA work at N = 256).
struct Tile {
    int kb, nb, W, pb, nkb, npb, N;
    double cost;
};

std::vector<Tile> tile_candidates(const G4Dims& d) {
    std::vector<Tile> out;
    for (int nb = 1; nb <= kMaxNb && nb <= d.Nw2; ++nb) {
        const int W = nb + d.Nwex - 1;
        if (W > kMaxW) break;
        const int r8 = (2 * W + 7) / 8 * 8;
        for (int kb = 1; kb <= d.Nc && 2 * kb * nb <= kARows; ++kb) {
            const int nkb = (d.Nc + kb - 1) / kb;
            for (int pb = 1; pb <= d.Nc; ++pb) {
                const int N = (2 * W * pb + 15) / 16 * 16;
                if (N > 256 || 2 * W * (pb - 1) + r8 > 256 || tc_smem_bytes(N, d.Nwex) > kSmemMax) break;
                const int npb = (d.Nc + pb - 1) / pb;
                const double cost = (double)nkb * npb * std::max((double)N, (128.0 + N) * 2.0 / 3.0) / nb;
                out.push_back(Tile{kb, nb, W, pb, nkb, npb, N, cost});
            }
        }
    }
    std::stable_sort(out.begin(), out.end(), [](const Tile& a, const Tile& b) { return a.cost < b.cost - 1e-9; });
    return out;
}

bool encode(const G4Dims& d, XtcPlan& X) {
    auto enc = encoder();
    if (!enc) return false;
    const cuuint64_t J = (cuuint64_t)X.J;
    const cuuint64_t es_b = X.f16 ? 2 : 4;      // element bytes
    const cuuint64_t dims[5] = {J, 2, (cuuint64_t)d.Nw2, (cuuint64_t)d.Nc, (cuuint64_t)X.gcap};
    const cuuint64_t strides[4] = {J * es_b, J * 2 * es_b, J * 2 * es_b * d.Nw2,
                                   J * 2 * es_b * d.Nw2 * d.Nc};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const cuuint32_t chunk = (cuuint32_t)chunk_of(X.f16);
    const cuuint32_t boxA[5] = {chunk, 2, (cuuint32_t)X.nb, (cuuint32_t)X.kb, 1};
    const cuuint32_t boxB[5] = {chunk, 2, (cuuint32_t)X.W, (cuuint32_t)X.pb, 1};
    CUtensorMap* maps[4] = {&X.mAh, &X.mAl, &X.mBh, &X.mBl};
    void* base[4] = {X.Xh, X.Xl, X.Xh, X.Xl};
    const CUtensorMapDataType dt = X.f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    for (int i = 0; i < 4; ++i) {
        CUresult r = enc(maps[i], dt, 5, base[i], dims, strides,
                         i < 2 ? boxA : boxB, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

template <typename T>
g4_status xalloc(g4_ctx* h, XtcPlan* X, T** p, size_t count) {
    const size_t bytes = count * sizeof(T);
    if (h->opt.mem_limit > 0 && h->bytes + bytes > (size_t)h->opt.mem_limit)
        return g4_fail(h, G4_ERR_OOM, "device memory limit reached (tensor-core exchange operands)");
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return g4_fail(h, G4_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) +
                                          " bytes failed (tensor-core exchange operands)");
    }
    h->bytes += bytes;
    X->held += bytes;
    return G4_OK;
}

template <bool F16>
cudaError_t raise_limits() {
    cudaError_t e;
    if ((e = raise_smem_limit(k_exchange_tc<0, 2, 4, F16>)) != cudaSuccess ||
        (e = raise_smem_limit(k_exchange_tc<1, 2, 4, F16>)) != cudaSuccess ||
        (e = raise_smem_limit(k_exchange_tc<0, 4, 12, F16>)) != cudaSuccess ||
        (e = raise_smem_limit(k_exchange_tc<1, 4, 12, F16>)) != cudaSuccess ||
        (e = raise_smem_limit(k_exchange_tc<0, 4, 16, F16>)) != cudaSuccess ||
        (e = raise_smem_limit(k_exchange_tc<1, 4, 16, F16>)) != cudaSuccess ||
        (e = raise_smem_limit(k_exchange_tc<0, 8, 16, F16>)) != cudaSuccess ||
        (e = raise_smem_limit(k_exchange_tc<1, 8, 16, F16>)) != cudaSuccess ||
        (e = raise_smem_limit(k_pack_xtc<F16>)) != cudaSuccess ||
        (e = raise_smem_limit(k_pack_xtc_M<F16, true>)) != cudaSuccess ||
        (e = raise_smem_limit(k_pack_xtc_M<F16, false>)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

using XKernel = void (*)(const __grid_constant__ CUtensorMap, const __grid_constant__ CUtensorMap,
                         const __grid_constant__ CUtensorMap, const __grid_constant__ CUtensorMap,
                         TParams);

// The kernel variant for a channel geometry (pp: reflected band), window and
// operand type: the register arrays of the epilogue hold the window W (WM >= W
// columns per momentum) and the transfers (2 NWH >= Nwex); the narrowest
// variant that fits does the least work per row.
template <bool F16>
XKernel pick(bool pp, bool w16, bool wide, bool narrow) {
    if (narrow) return pp ? k_exchange_tc<1, 2, 4, F16> : k_exchange_tc<0, 2, 4, F16>;
    if (wide) return pp ? k_exchange_tc<1, 8, 16, F16> : k_exchange_tc<0, 8, 16, F16>;
    return pp ? (w16 ? k_exchange_tc<1, 4, 16, F16> : k_exchange_tc<1, 4, 12, F16>)
              : (w16 ? k_exchange_tc<0, 4, 16, F16> : k_exchange_tc<0, 4, 12, F16>);
}

}  // namespace

// Largest X buffer (both planes) a handle allocates; problems whose operands
// exceed it are processed in several groups of diagonals per batch, of equal
// size.  A deferred handle holds no batch of G (the size of X again) and
// forms each group from M, reading M once per group, so it takes a larger X.
constexpr size_t kXBudget = (size_t)12 << 30;
constexpr size_t kXBudgetDeferred = (size_t)96 << 30;

bool xtc_feasible(const G4Dims& d) {
    return d.Nwex <= kMaxW && !tile_candidates(d).empty();
}

namespace {

// Work lists, tensor maps and shared memory of one tile shape (the X buffers,
// diagonal list and groups do not depend on it).
g4_status build_tiling(g4_ctx* h, XtcPlan* X, const Tile& t) {
    const G4Dims& d = h->d;
    X->kb = t.kb;
    X->nb = t.nb;
    X->W = t.W;
    X->pb = t.pb;
    X->nkb = t.nkb;
    X->npb = t.npb;
    X->N = t.N;
    X->gw0.clear();
    X->gwn.clear();
    X->gd0.clear();
    X->gdn.clear();
    X->gs0.clear();
    X->gsn.clear();
    // groups of whole items; the work list of a group follows its diagonals
    // the entries of D = 0 (split tiles, sixteen times the epilogue work of a
    // tile) get a launch of their own with one tile per block, so that they
    // spread over the GPU instead of loading the few blocks of one run
    std::vector<int4> work, swork;
    int pos = 0;
    for (size_t it = 0; it < X->itemlen.size();) {
        const int g0 = pos;
        const int w0 = (int)work.size();
        const int s0 = (int)swork.size();
        while (it < X->itemlen.size() && pos + X->itemlen[it] - g0 <= X->gcap) {
            const int len = X->itemlen[it];
            for (int u = 0; u < len; ++u) {
                const int a = pos + u - g0;
                const int b = len == 2 ? (pos + (1 - u) - g0) : a;
                const int dk = X->dl[pos + u].x, dn = X->dl[pos + u].y;
                const int nlo = std::max(0, -dn), nhi = std::min(d.Nw2, d.Nw2 - dn);
                const bool split = dk == 0 && dn == 0;
                for (int n0 = nlo; n0 < nhi; n0 += X->nb) {
                    if (split)
                        swork.push_back(make_int4(a | (b << 16), dk, dn, n0 | (1 << 10)));
                    else
                        work.push_back(make_int4(a | (b << 16), dk, dn, n0));
                }
            }
            pos += len;
            ++it;
        }
        X->gd0.push_back(g0);
        X->gdn.push_back(pos - g0);
        X->gw0.push_back(w0);
        X->gwn.push_back((int)work.size() - w0);
        X->gs0.push_back(s0);
        X->gsn.push_back((int)swork.size() - s0);
    }
    const size_t nmain = work.size();
    work.insert(work.end(), swork.begin(), swork.end());  // split entries after the main ones
    for (size_t g = 0; g < X->gs0.size(); ++g) X->gs0[g] += (int)nmain;
    if (X->work) {
        cudaFree(X->work);
        X->work = nullptr;
        h->bytes -= std::min(h->bytes, X->work_bytes);
        X->held -= std::min(X->held, X->work_bytes);
    }
    g4_status st;
    if ((st = xalloc(h, X, &X->work, work.size())) != G4_OK) return st;
    X->work_bytes = work.size() * sizeof(int4);
    cudaError_t e = cudaMemcpy(X->work, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange work list upload");
    if (!encode(d, *X))
        return g4_fail(h, G4_ERR_CUDA, "cuTensorMapEncodeTiled failed for the exchange operands");
    // at least 116 KB, so that two blocks never share an SM (each holds all 512
    // tensor-memory columns)
    X->smem = std::max(tc_smem_bytes(X->N, d.Nwex), 116 * 1024);
    return G4_OK;
}

// Tile shapes chosen by timing, per process (and in the file named by
// G4_TUNE_CACHE): key = GPU model and problem shape, value = "kb,nb,pb".
std::mutex g_xt_mu;
std::map<std::string, std::array<int, 3>> g_xt;

std::string xt_key(const g4_ctx* h, bool f16) {
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) name = prop.name;
    for (char& c : name)
        if (c == ' ' || c == '=') c = '_';
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|xtc%s|ch%d|Nc%d|Lx%d|Nw2_%d|Nwex%d|m0_%d|Nkex%d|b%d", name.c_str(),
                  f16 ? "16" : "32", h->d.ch, h->d.Nc, h->d.Lx, h->d.Nw2, h->d.Nwex, h->d.m0, h->d.Nkex,
                  h->batch);
    return buf;
}

bool xt_lookup(const std::string& key, std::array<int, 3>* out) {
    std::lock_guard<std::mutex> lock(g_xt_mu);
    auto it = g_xt.find(key);
    if (it != g_xt.end()) {
        *out = it->second;
        return true;
    }
    const char* path = std::getenv("G4_TUNE_CACHE");
    FILE* f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        char* eq = std::strchr(line, '=');
        if (!eq) continue;
        *eq = 0;
        std::array<int, 3> v{};
        if (key == line && std::sscanf(eq + 1, "%d,%d,%d", &v[0], &v[1], &v[2]) == 3) {
            *out = v;
            found = true;
        }
    }
    std::fclose(f);
    if (found) g_xt[key] = *out;
    return found;
}

void xt_store(const std::string& key, const std::array<int, 3>& v) {
    std::lock_guard<std::mutex> lock(g_xt_mu);
    g_xt[key] = v;
    const char* path = std::getenv("G4_TUNE_CACHE");
    FILE* f = path ? std::fopen(path, "a") : nullptr;
    if (!f) return;
    std::fprintf(f, "%s=%d,%d,%d\n", key.c_str(), v[0], v[1], v[2]);
    std::fclose(f);
}

constexpr int kTuneCandidates = 4;

}  // namespace

g4_status xtc_prepare(g4_ctx* h) {
    const G4Dims& d = h->d;
    XtcPlan* X = new (std::nothrow) XtcPlan();
    if (!X) return g4_fail(h, G4_ERR_OOM, "host allocation of the exchange plan");
    h->xtc = X;
    const std::vector<Tile> cands = d.Nwex <= kMaxW ? tile_candidates(d) : std::vector<Tile>();
    if (cands.empty()) return g4_fail(h, G4_ERR_INVALID, "no tensor-core exchange tiling for these sizes");
    X->f16 = h->opt.operands == G4_OPERANDS_FP16;
    X->Jh = h->Bp;
    X->J = 2 * h->Bp;
    if (X->Jh % chunk_of(X->f16) != 0)
        return g4_fail(h, G4_ERR_INVALID, "padded batch is not a whole number of operand chunks");
    X->aoff = (d.ch == G4_PH_TRANSVERSE || d.ch == G4_PP_UPDOWN) ? X->Jh / chunk_of(X->f16) : 0;

    // diagonals in pairs (D, -D), so that a diagonal read as A is read as B soon after
    std::vector<int> ksub((size_t)d.Nc * d.Nc);
    for (int a = 0; a < d.Nc; ++a)
        for (int b = 0; b < d.Nc; ++b) {
            const int ax = a % d.Lx, ay = a / d.Lx, bx = b % d.Lx, by = b / d.Lx;
            ksub[a * d.Nc + b] = (ax - bx + d.Lx) % d.Lx + d.Lx * ((ay - by + d.Ly) % d.Ly);
        }
    for (int dn = 0; dn < d.Nw2; ++dn)
        for (int dk = 0; dk < d.Nc; ++dk) {
            const int mk = ksub[0 * d.Nc + dk];
            if (dn == 0) {
                if (mk < dk) continue;
                X->dl.push_back(make_int2(dk, 0));
                if (mk != dk) {
                    X->dl.push_back(make_int2(mk, 0));
                    X->itemlen.push_back(2);
                } else {
                    X->itemlen.push_back(1);
                }
            } else {
                X->dl.push_back(make_int2(dk, dn));
                X->dl.push_back(make_int2(mk, -dn));
                X->itemlen.push_back(2);
            }
        }
    // one diagonal of the group, both planes
    const size_t per_slot = (size_t)d.Nc * d.Nw2 * 2 * X->J * (X->f16 ? 2 : 4) * 2;
    size_t budget = h->deferred ? kXBudgetDeferred : kXBudget;
    if (h->opt.mem_limit > 0) {
        const size_t left = (size_t)h->opt.mem_limit > h->bytes ? (size_t)h->opt.mem_limit - h->bytes : 0;
        budget = std::min(budget, left);
    }
    const size_t fit = budget / per_slot;
    if (fit < 2) return g4_fail(h, G4_ERR_OOM, "no room for the tensor-core exchange operands");
    const size_t ngroups = (X->dl.size() + fit - 1) / fit;
    X->gcap = (int)std::min<size_t>(fit, ((X->dl.size() + ngroups - 1) / ngroups + 1) / 2 * 2);
    g4_status st;
    X->xbytes = (size_t)X->gcap * per_slot;
    if ((st = xalloc(h, X, (char**)&X->Xh, X->xbytes / 2)) != G4_OK) return st;
    if ((st = xalloc(h, X, (char**)&X->Xl, X->xbytes / 2)) != G4_OK) return st;
    if ((st = xalloc(h, X, &X->dlist, X->dl.size())) != G4_OK) return st;
    cudaError_t e = cudaMemcpy(X->dlist, X->dl.data(), X->dl.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange diagonal list upload");
    if (h->deferred) {
        // the pack finds a diagonal's position by the list's arithmetic
        // (diag_pos) with a table for dn = 0; check it against the list
        std::vector<int> pos0(d.Nc, -1);
        for (size_t p = 0; p < X->dl.size(); ++p)
            if (X->dl[p].y == 0) pos0[X->dl[p].x] = (int)p;
        for (int p = 0; p < (int)X->dl.size(); ++p) {
            const int dk = X->dl[p].x, dn = X->dl[p].y;
            const int dkx = dk % d.Lx, dky = dk / d.Lx;
            const int mk = (d.Lx - dkx) % d.Lx + d.Lx * ((d.Ly - dky) % d.Ly);
            const int q = dn > 0 ? d.Nc + (dn - 1) * 2 * d.Nc + 2 * dk
                                 : dn < 0 ? d.Nc + (-dn - 1) * 2 * d.Nc + 2 * mk + 1 : pos0[dk];
            if (q != p) return g4_fail(h, G4_ERR_INVALID, "diagonal list order (internal)");
        }
        if (d.Nc > 256) return g4_fail(h, G4_ERR_INVALID, "deferred staging takes at most 256 momenta");
        if ((st = xalloc(h, X, &X->pos0, pos0.size())) != G4_OK) return st;
        if ((st = xalloc(h, X, &X->g0f, (size_t)2 * d.N)) != G4_OK) return st;
        e = cudaMemcpy(X->pos0, pos0.data(), pos0.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange diagonal index upload");
        // the persistent pack from M: one block per SM
        const bool m64 = h->opt.m_complex64 != 0;
        auto* pk = X->f16 ? (m64 ? k_pack_xtc_M<true, true> : k_pack_xtc_M<true, false>)
                          : (m64 ? k_pack_xtc_M<false, true> : k_pack_xtc_M<false, false>);
        if ((e = raise_smem_limit(pk)) != cudaSuccess) return g4_cuda_fail(h, e, "pack smem attribute");
        const int et = m64 ? 128 : 64, sl = X->f16 ? 32 : 16;
        const int cj = d.Nw2 < et ? d.Nw2 : et, ri = d.Nw2 < et ? et / d.Nw2 : 1;
        const long long ntiles = (long long)d.Nc * d.Nc * ((d.Nw2 + ri - 1) / ri) *
                                 ((d.Nw2 + cj - 1) / cj) * (X->Jh / sl);
        const int per_sm = 1;
        X->packm_grid = (int)std::min<long long>(ntiles, (long long)num_sms() * per_sm);
    }
    X->pack_smem = X->J * (kPackN + 1) * (int)sizeof(float2);
    e = X->f16 ? raise_limits<true>() : raise_limits<false>();
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange smem attribute");

    // The tile shape: the cost model's choice, or -- with autotuning on and no
    // short wait budget -- the fastest of its best few candidates, each timed
    // over one full batch on the handle's own buffers (the staged G is still
    // all zero, so the accumulator, cleared when the handle is made, is left
    // unchanged), best of two after a warm-up.
    Tile best = cands[0];
    const bool tune = h->opt.autotune && h->opt.timeout_cycles == 0 && cands.size() > 1;
    if (tune) {
        const std::string key = xt_key(h, X->f16);
        std::array<int, 3> v{};
        bool known = xt_lookup(key, &v);
        if (known) {
            known = false;
            for (const Tile& t : cands)
                if (t.kb == v[0] && t.nb == v[1] && t.pb == v[2]) {
                    best = t;
                    known = true;
                }
        }
        if (!known) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
                if (e0) cudaEventDestroy(e0);
                return g4_cuda_fail(h, cudaGetLastError(), "autotune events");
            }
            const bool prof = h->prof_on;
            h->prof_on = false;
            float best_ms = 1e30f;
            const int n = std::min<int>(kTuneCandidates, (int)cands.size());
            for (int c = 0; c < n && st == G4_OK; ++c) {
                if ((st = build_tiling(h, X, cands[c])) != G4_OK) break;
                float ms = 1e30f;
                for (int rep = 0; rep < 3 && st == G4_OK; ++rep) {
                    cudaEventRecord(e0, h->stream);
                    // (a deferred handle has no staged M: its pack writes zero planes)
                    st = xtc_run(h, h->deferred ? 0 : h->batch);
                    cudaEventRecord(e1, h->stream);
                    float t = 0.f;
                    if (st == G4_OK && cudaEventSynchronize(e1) == cudaSuccess &&
                        cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && rep > 0)
                        ms = std::min(ms, t);
                }
                if (st == G4_OK && ms < best_ms) {
                    best_ms = ms;
                    best = cands[c];
                }
            }
            h->prof_on = prof;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (st != G4_OK) return st;
            xt_store(key, {best.kb, best.nb, best.pb});
        }
    }
    return build_tiling(h, X, best);
}

g4_status xtc_run(g4_ctx* h, int staged) {
    const XtcPlan* X = (const XtcPlan*)h->xtc;
    const G4Dims& d = h->d;
    TParams P;
    P.acc = h->acc;
    P.status = h->dstatus;
    P.Lx = d.Lx;
    P.Ly = d.Ly;
    P.mLx = (uint32_t)(((1u << 24) + d.Lx - 1) / d.Lx);
    P.Nc = d.Nc;
    P.Nw2 = d.Nw2;
    P.N = d.N;
    P.Nwex = d.Nwex;
    P.Nkex = d.Nkex;
    P.NQ = d.NQ;
    P.m0 = d.m0;
    P.kb = X->kb;
    P.nb = X->nb;
    P.W = X->W;
    P.pb = X->pb;
    P.nkb = X->nkb;
    P.npb = X->npb;
    P.nchunk = X->J / chunk_of(X->f16);
    P.aoff = X->aoff;
    P.bplane = X->N * kRowBytes;
    // per stage: A hi and lo boxes (2 components x nb x kb rows of 128 bytes), B likewise
    P.txbytes = (uint32_t)(2 * (kRowBytes * 2 * X->nb * X->kb) + 2 * (kRowBytes * 2 * X->W * X->pb));
    P.idesc = X->f16 ? idesc_f16(kARows, X->N) : idesc_tf32(kARows, X->N);
    P.gmax = h->deferred ? h->gscale : h->gmax;
    P.pair = h->opt.accum == G4_ACCUM_F32PAIR;
    P.budget = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : 4000000000LL;
    // deferred staging: the G0 all staged measurements share, if they do
    const double2* g0s = nullptr;
    if (h->deferred && staged > 0) {
        g0s = h->slots->s[0].G0;
        for (int r = 1; r < staged && g0s; ++r)
            if (h->slots->s[r].G0 != g0s) g0s = nullptr;
        if (g0s) {
            k_g0_narrow<<<(2 * d.N + 255) / 256, 256, 0, h->stream>>>(g0s, X->g0f, 2 * d.N);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return g4_cuda_fail(h, e, "G0 narrowing launch");
        }
    }
    for (size_t g = 0; g < X->gd0.size(); ++g) {
        prof_begin(h, G4_K_PACK_EXCHANGE);
        if (h->deferred) {
            // FP16 pairs: pack with the kept scale, check it against the
            // batch's largest component, pack again only if it had to change
            const bool m64 = h->opt.m_complex64 != 0;
            auto* pack = X->f16 ? (m64 ? k_pack_xtc_M<true, true> : k_pack_xtc_M<true, false>)
                                : (m64 ? k_pack_xtc_M<false, true> : k_pack_xtc_M<false, false>);
            const int smem = X->f16 ? (m64 ? PackM<true, true>::SMEM : PackM<true, false>::SMEM)
                                    : (m64 ? PackM<false, true>::SMEM : PackM<false, false>::SMEM);
            // the direct term's operands go into the window with the planes
            DirectOut D{};
            if (has_direct(d.ch)) {
                direct_window_ptrs(h, &D.araw, &D.braw, &D.wmax, &D.w0, &D.Bw);
                D.ws = d.ch == G4_PH_DENSITY ? 1.f : -1.f;
            }
            cudaError_t e = cudaSuccess;
            if (X->f16) e = cudaMemsetAsync(h->gmax, 0, sizeof(unsigned), h->stream);
            for (int pass = 0; pass < (X->f16 ? 2 : 1) && e == cudaSuccess; ++pass) {
                pack<<<X->packm_grid, 544, smem, h->stream>>>(
                    *h->slots, staged, X->Jh, g0s ? X->g0f : nullptr, X->pos0, X->gd0[g], X->gdn[g], X->Xh, X->Xl,
                    h->gscale, pass == 0 && X->f16 ? h->gmax : nullptr, pass ? h->gredo : nullptr, D, d,
                    P.budget, h->dstatus);
                if (pass == 0 && X->f16) k_scale_check<<<1, 32, 0, h->stream>>>(h->gmax, h->gscale, h->gredo);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange pack launch");
        } else {
            auto* pack = X->f16 ? k_pack_xtc<true> : k_pack_xtc<false>;
            pack<<<dim3(d.Nc, X->gdn[g], (d.Nw2 + kPackN - 1) / kPackN), 256, X->pack_smem, h->stream>>>(
                h->Gd, staged, X->Jh, X->dlist + X->gd0[g], X->Xh, X->Xl, h->gmax, d);
        }
        prof_end(h, G4_K_PACK_EXCHANGE);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange pack launch");
        const bool pp = d.ch == G4_PP_UPDOWN, w16 = X->W > 12, wide = d.Nwex > 8;
        const bool narrow = X->W <= 4 && d.Nwex <= 4;
        XKernel kern = X->f16 ? pick<true>(pp, w16, wide, narrow) : pick<false>(pp, w16, wide, narrow);
        // main tiles in runs of two row-frequency blocks of one diagonal, then
        // the split tiles of D = 0 one per block
        for (int part = 0; part < 2; ++part) {
            const int w0 = part ? X->gs0[g] : X->gw0[g], wn = part ? X->gsn[g] : X->gwn[g];
            // a deferred handle's group (all diagonals at once) is launched in
            // six pieces of its work list (runs of two entries stay whole):
            // measured faster than one launch on c64_w64 (33.3 against 34.6 ms
            // per batch); on c36_w64's single group one launch is faster
            const int pieces = (part == 0 && h->deferred && X->gd0.size() == 1) ? 6 : 1;
            const int wstep = ((wn + pieces - 1) / pieces + 1) / 2 * 2;
            for (int c0 = 0; c0 < wn; c0 += (wstep > 0 ? wstep : wn)) {
                const int wc = std::min(wn - c0, wstep > 0 ? wstep : wn);
                P.work = X->work + w0 + c0;
                P.ntiles = wc * X->nkb * X->npb;
                if (P.ntiles == 0) continue;
                P.run = part ? 1 : 2 * X->nkb * X->npb;
                const int grid = std::min((P.ntiles + P.run - 1) / P.run, num_sms());
                prof_begin(h, G4_K_EXCHANGE);
                kern<<<grid, kThreads, X->smem, h->stream>>>(X->mAh, X->mAl, X->mBh, X->mBl, P);
                prof_end(h, G4_K_EXCHANGE);
                e = cudaGetLastError();
                if (e != cudaSuccess) return g4_cuda_fail(h, e, "tensor-core exchange launch");
            }
        }
    }
    return G4_OK;
}

void xtc_release(g4_ctx* h) {
    XtcPlan* X = (XtcPlan*)h->xtc;
    if (!X) return;
    void* ptrs[] = {X->Xh, X->Xl, X->work, X->dlist, X->pos0, X->g0f};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    h->bytes -= std::min(h->bytes, X->held);
    delete X;
    h->xtc = nullptr;
}
