// Exchange term of the particle-hole magnetic G4 update (the second product
// of the accumulation of Eq. (1), Sec. 2.1, in this channel):
//
//   Exc(K1, K2, Q) = sum_r s_r sum_s G_s(K2, K1) G_s(K1+Q, K2+Q).
//
// For a fixed difference D = K2 - K1 = (dk, dn) this is a banded outer
// product over the batch index j = (r, s):
//
//   Exc(K1, K1+D, Q) = sum_j u_j(K1) w_j(K1+Q),
//   u_j(K1) = G~_s(K1+D, K1)      (the D-th diagonal of G~, indexed by column)
//   w_j(P)  = G~_s(P, P+D)        (the -D-th diagonal, indexed by column P+D)
//
// with G~ = sqrt(s_r) G as written by the G build, so u w carries s_r.  A
// thread owns one momentum pair (k1, q) and a window of TN frequencies n1
// times MW transfers m: TN + (TN+MW-1) complex shared-memory loads per j feed
// TN*MW complex multiply-adds (register tiling).  Threads of a warp share
// p = k1 (+) q, so their w loads are broadcasts.
//
// Staging: one thread issues TMA copies of the diagonal-major G~ (complex64)
// into a 3-deep shared-memory ring guarded by mbarriers (bounded waits):
//   u: box (TN+2 frequencies, all Nc momenta, JC batch entries) -- the +2
//      pads each row to a bank-conflict-free stride;
//   w: one box (TN+MW frequencies, JC entries) per momentum p of the block,
//      started at an even frequency (16-byte aligned coordinate); columns
//      outside the grid are zero-filled by the copy.
// FP32 accumulation over the batch, then one FP64 read-modify-write of the
// accumulator: acc[K1][K2][q][m] -= Exc.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "g4_internal.h"

namespace {

constexpr int kMaxThreads = 192;   // pairs per block (two blocks per SM)
constexpr int kRing = 3;

struct XParams {
    const int* pairs;      // (k1 | q << 16), sorted by p = k1 (+) q
    const int* kadd;
    const int* ksub;
    const int2* work;      // (dnI, window) pairs with a non-empty n1 range
    double2* acc;
    unsigned* status;
    G4Dims d;
    int npairs;
    int nj;                // 2 * staged
    int nmc;               // m chunks
    int JC;                // j per stage
    int uBytes;            // one u stage (128-byte aligned)
    int wBytes;            // one w row block per p (128-byte aligned)
    int nPmax;
    long long budget;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ float4 lds128(uint32_t addr) {
    float4 v;
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "r"(addr));
    return v;
}

__device__ __forceinline__ void tma_5d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                       int c1, int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

// Variants: kSame (magnetic, density) pairs u and w of the same spin over the
// shifted band P = K1+Q; kCross (transverse) pairs u of spin -s with w of spin
// s; kPP (particle-particle, Eq. (1)) pairs opposite spins over the reflected
// band P = Q-K1 (w index decreasing with n1) and adds instead of subtracting.
enum { kSame = 0, kPP = 1, kCross = 3 };

template <int TN, int MW, int WOFF, int V>
__global__ void __launch_bounds__(kMaxThreads, 3)
    k_exchange(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmW,
               XParams P) {
    constexpr int UW = TN + 2;              // u row (complex); UW/2 odd: conflict-free 16-byte loads
    constexpr int WW = (TN + MW + 1) & ~1;  // w row (complex): TN+MW-1 needed + alignment slack
    extern __shared__ __align__(128) uint8_t smem_raw[];
    const G4Dims& d = P.d;
    const int Nw2 = d.Nw2, Nc = d.Nc;

    const int dk = blockIdx.z / P.nmc, mc = blockIdx.z - dk * P.nmc;
    const int m0 = mc * MW;
    const int2 wk = P.work[blockIdx.y];
    const int dnI = wk.x, a = wk.y * TN;
    const int dn = dnI - (Nw2 - 1);
    const int lo = max(a, max(0, -dn)), hi = min(a + TN, min(Nw2, Nw2 - dn));

    const int pi0 = blockIdx.x * blockDim.x;
    const int pi = pi0 + threadIdx.x;
    const bool active = pi < P.npairs;
    const int plast = min(P.npairs, pi0 + (int)blockDim.x) - 1;
    const int pair0 = P.pairs[pi0], pairL = P.pairs[plast];
    // sort key of a pair (the momentum of its w row before the diagonal shift)
    auto key = [&](int pr) {
        const int kk = pr & 0xffff, qq = pr >> 16;
        return V == kPP ? P.ksub[qq * Nc + kk] : P.kadd[kk * Nc + qq];
    };
    const int pfirst = key(pair0);
    const int nP = key(pairL) - pfirst + 1;

    int k1 = 0, q = 0, pl = 0;
    if (active) {
        const int pr = P.pairs[pi];
        k1 = pr & 0xffff;
        q = pr >> 16;
        pl = key(pr) - pfirst;
    }
    const int dkn = P.ksub[dk];                  // (-)dk
    const int dnIneg = 2 * (Nw2 - 1) - dnI;      // diagonal -dn
    // even start of the w window: columns a+m0+dn .. (shifted band) or
    // m0 + Nw2-1 - (a+TN-1) .. (reflected band, frequency of Q-K1)
    const int wx0 = (V == kPP ? m0 + Nw2 - a - TN : a + m0 + dn) - WOFF;
    // A copy's innermost coordinate must be 16-byte aligned (even, for 8-byte
    // elements).  Planning guarantees it; a block that would violate it records
    // the fault and does nothing.
    if (((wx0 | a) & 1) != 0) {
        if (threadIdx.x == 0) atomicOr(P.status, (unsigned)G4_DEV_BADARG);
        return;
    }

    const int stageBytes = P.uBytes + P.nPmax * P.wBytes;
    uint8_t* ring = smem_raw;
    uint64_t* full = (uint64_t*)(smem_raw + kRing * stageBytes);
    uint64_t* empty = full + kRing;                // one arrival per warp when a stage is consumed
    int* wrow = (int*)(empty + kRing);             // [nP] w-row momenta p (+) dk
    const int nwarps = blockDim.x >> 5;
    __shared__ int abort_flag;

    const int nstages = (P.nj + P.JC - 1) / P.JC;
    for (int pp = threadIdx.x; pp < nP; pp += blockDim.x)
        wrow[pp] = V == kPP ? pfirst + pp : P.kadd[(pfirst + pp) * Nc + dk];
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < kRing; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])),
                         "r"(nwarps));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int st) {
        const int s = st % kRing;
        const int j0 = st * P.JC;
        const uint32_t base = smem_u32(ring + s * stageBytes);
        const uint32_t bytes = (uint32_t)(P.JC * Nc * UW * 8 + nP * P.JC * WW * 8);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         smem_u32(&full[s])),
                     "r"(bytes)
                     : "memory");
        // coordinates (n, k, dnI, dk, j)
        tma_5d(base, &tmU, &full[s], a, 0, dnI, dk, j0);
        for (int pp = 0; pp < nP; ++pp)
            tma_5d(base + P.uBytes + pp * P.wBytes, &tmW, &full[s], wx0, wrow[pp], dnIneg, dkn, j0);
    };

    int issued = 0;  // stages whose copies thread 0 has started
    if (threadIdx.x == 0) {
        for (int st = 0; st < kRing - 1 && st < nstages; ++st) issue(st);
        issued = min(kRing - 1, nstages);
    }

    float2 acc[TN][MW];
#pragma unroll
    for (int t = 0; t < TN; ++t)
#pragma unroll
        for (int mm = 0; mm < MW; ++mm) acc[t][mm] = make_float2(0.f, 0.f);

    for (int st = 0; st < nstages; ++st) {
        const int s = st % kRing;
        if (threadIdx.x == 0 && st + kRing - 1 < nstages && !abort_flag) {
            // the buffer refilled now was last read in stage st-1: wait until every warp is done
            if (st >= 1) {
                const int sp = (st - 1) % kRing;
                const long long t0 = clock64();
                while (!mbar_try(&empty[sp], ((st - 1) / kRing) & 1)) {
                    if (clock64() - t0 > P.budget) {
                        abort_flag = 1;
                        break;
                    }
                }
            }
            if (!abort_flag) {
                issue(st + kRing - 1);
                issued = st + kRing;
            }
        }
        {
            const long long t0 = clock64();
            while (!mbar_try(&full[s], (st / kRing) & 1)) {
                if (abort_flag) break;
                if (clock64() - t0 > P.budget) {
                    abort_flag = 1;
                    break;
                }
            }
        }
        if (abort_flag) break;
        const int jc = min(P.JC, P.nj - st * P.JC);
        // 32-bit shared-window addresses: the operand reads are explicit ld.shared
        const uint32_t su = smem_u32(ring + s * stageBytes) + (uint32_t)(k1 * UW * 8);
        const uint32_t sw = smem_u32(ring + s * stageBytes + P.uBytes + pl * P.wBytes);
        const uint32_t ustep = (uint32_t)(Nc * UW * 8), wstep = (uint32_t)(WW * 8);
        if (active) {
#pragma unroll 1
            for (int jj = 0; jj < jc; ++jj) {
                const uint32_t ur = su + (V == kSame ? jj : (jj ^ 1)) * ustep;
                const uint32_t wr = sw + jj * wstep;
                // w[i] = element i of the row (aligned pairs); the thread's window starts at WOFF
                float2 w[WW];
#pragma unroll
                for (int i = 0; i < WW / 2; ++i) {
                    const float4 v = lds128(wr + 16 * i);
                    w[2 * i] = make_float2(v.x, v.y);
                    w[2 * i + 1] = make_float2(v.z, v.w);
                }
#pragma unroll
                for (int t2 = 0; t2 < TN / 2; ++t2) {
                    const float4 uv = lds128(ur + 16 * t2);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int t = 2 * t2 + h;
                        const float2 x = h ? make_float2(uv.z, uv.w) : make_float2(uv.x, uv.y);
#pragma unroll
                        for (int mm = 0; mm < MW; ++mm) {
                            const float2 y = w[(V == kPP ? TN - 1 - t : t) + mm + WOFF];
                            acc[t][mm].x = fmaf(x.x, y.x, acc[t][mm].x);
                            acc[t][mm].y = fmaf(x.x, y.y, acc[t][mm].y);
                            acc[t][mm].x = fmaf(-x.y, y.y, acc[t][mm].x);
                            acc[t][mm].y = fmaf(x.y, y.x, acc[t][mm].y);
                        }
                    }
                }
            }
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s]))
                         : "memory");
    }
    __syncthreads();
    if (abort_flag) {
        if (threadIdx.x == 0) {
            atomicOr(P.status, (unsigned)G4_DEV_TIMEOUT);
            // let this block's copies already in flight land before it exits (bounded)
            for (int st = (issued > kRing ? issued - kRing : 0); st < issued; ++st) {
                const long long t0 = clock64();
                while (!mbar_try(&full[st % kRing], (st / kRing) & 1) && clock64() - t0 < kDrainBudget) {
                }
            }
        }
        return;
    }
    // Epilogue through shared memory (the ring is free now): every thread parks
    // its TN x MW sums, then each warp instruction updates 32/MW runs of MW
    // consecutive m values (MW*16 contiguous bytes each) instead of 32
    // scattered entries.
    constexpr int PS = TN * MW + 1;                                // padded per-thread stride
    float2* park = (float2*)ring;                                  // [blockDim][PS]
    size_t* rowbase = (size_t*)(ring + (size_t)blockDim.x * PS * sizeof(float2) + 8);
    if (active) {
        const int k2 = P.kadd[k1 * Nc + dk];
        const size_t K1 = (size_t)k1 * Nw2 + a, K2 = (size_t)k2 * Nw2 + a + dn;
        rowbase[threadIdx.x] = (K1 * d.N + K2) * d.NQ + (size_t)q * d.Nwex + m0;
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
            for (int mm = 0; mm < MW; ++mm) park[threadIdx.x * PS + t * MW + mm] = acc[t][mm];
    }
    __syncthreads();
    const int nact = min((int)blockDim.x, P.npairs - pi0);
    const int runs = nact * TN;                    // (pair, t) runs of MW entries
    const int mmax = min(MW, d.Nwex - m0);
    const size_t tstride = (size_t)(d.N + 1) * d.NQ;  // K1+1, K2+1
    // loads of a batch are issued before its stores (a store could alias a later
    // load, so the compiler would otherwise serialise every round trip)
    constexpr int kB = 8;
    const int total = runs * MW;
    for (int e0 = threadIdx.x; e0 < total; e0 += kB * blockDim.x) {
        double2* ptr[kB];
        double2 old[kB];
        float2 v[kB];
        bool ok[kB];
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            const int e = e0 + i * blockDim.x;
            const int mm = e % MW, r = e / MW;
            const int pr = r / TN, t = r - pr * TN;
            const int n1 = a + t;
            ok[i] = e < total && mm < mmax && n1 >= lo && n1 < hi;
            ptr[i] = P.acc + (ok[i] ? rowbase[pr] + (size_t)t * tstride + mm : 0);
            v[i] = ok[i] ? park[pr * PS + t * MW + mm] : make_float2(0.f, 0.f);
            if (V == kPP) v[i] = make_float2(-v[i].x, -v[i].y);  // this channel adds
        }
#pragma unroll
        for (int i = 0; i < kB; ++i)
            if (ok[i]) old[i] = *ptr[i];
#pragma unroll
        for (int i = 0; i < kB; ++i)
            if (ok[i]) *ptr[i] = make_double2(old[i].x - (double)v[i].x, old[i].y - (double)v[i].y);
    }
}

struct XPlan {
    CUtensorMap tmU, tmW;
    int2* work = nullptr;
    int nwork = 0, nwork_even = 0;   // work items with an even w start come first
    int TN = 8, MW = 8;
    int JC = 1, uBytes = 0, wBytes = 0, nPmax = 1;
    int chunk = 32;                  // pairs (threads) per block
    int V = 0;                       // kernel variant (channel)
    size_t smem = 0;
};

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

inline int align128(int x) { return (x + 127) & ~127; }

// Largest dynamic shared memory a plan may ask for (the device opt-in limit
// less the kernel's small static part); the per-function limit is raised to
// the device maximum once, since every handle shares it.
constexpr int kMaxSmem = 227 * 1024 - 1024;

template <int TN, int MW, int V>
cudaError_t set_smem_v() {
    cudaError_t e = raise_smem_limit(k_exchange<TN, MW, 0, V>);
    if (e != cudaSuccess || V == kPP) return e;
    return raise_smem_limit(k_exchange<TN, MW, 1, V>);
}

template <int TN, int MW>
cudaError_t set_smem(int V) {
    return V == kPP ? set_smem_v<TN, MW, kPP>()
                    : (V == kCross ? set_smem_v<TN, MW, kCross>() : set_smem_v<TN, MW, kSame>());
}

// The w window of a block starts at column a + m0 + dn; its parity (uniform over
// the launch only when dn has fixed parity) selects the instantiation.  Windows
// of both parities are handled by two launches over the split work list.
template <int TN, int MW, int V>
void launch_v(const XPlan& X, XParams P, dim3 grid, cudaStream_t s) {
    if (V == kPP) {
        // reflected band: the window start m0 + Nw2 - a - TN is always even
        grid.y = X.nwork;
        if (grid.y) k_exchange<TN, MW, 0, V><<<grid, X.chunk, X.smem, s>>>(X.tmU, X.tmW, P);
        return;
    }
    P.work = X.work;
    grid.y = X.nwork_even;
    if (grid.y) k_exchange<TN, MW, 0, V><<<grid, X.chunk, X.smem, s>>>(X.tmU, X.tmW, P);
    P.work = X.work + X.nwork_even;
    grid.y = X.nwork - X.nwork_even;
    if (grid.y) k_exchange<TN, MW, 1, V><<<grid, X.chunk, X.smem, s>>>(X.tmU, X.tmW, P);
}

template <int TN, int MW>
void launch(const XPlan& X, XParams P, dim3 grid, cudaStream_t s) {
    if (X.V == kPP) launch_v<TN, MW, kPP>(X, P, grid, s);
    else if (X.V == kCross) launch_v<TN, MW, kCross>(X, P, grid, s);
    else launch_v<TN, MW, kSame>(X, P, grid, s);
}

int variant_of(int ch) {
    return ch == G4_PP_UPDOWN ? kPP : (ch == G4_PH_TRANSVERSE ? kCross : kSame);
}

}  // namespace

// ---------------------------------------------------------------- planning

namespace {

// One launch configuration: register tile (32/MW n1 x MW m), block size, stage
// sizes, work list and tensor maps.
g4_status make_plan(g4_ctx* h, int MW, int chunk_cap, const std::vector<int>& pofs, XPlan* X) {
    const G4Dims& d = h->d;
    X->MW = MW;
    X->TN = 32 / MW;
    X->V = variant_of(d.ch);
    const int TN = X->TN;
    // balanced blocks of at most chunk_cap pairs, a multiple of 32
    {
        const int nch = (h->npairs + chunk_cap - 1) / chunk_cap;
        const int per = (h->npairs + nch - 1) / nch;
        X->chunk = std::min(chunk_cap, (per + 31) / 32 * 32);
    }
    X->nPmax = 1;
    for (int c = 0; c < h->npairs; c += X->chunk) {
        const int last = std::min(h->npairs, c + X->chunk) - 1;
        X->nPmax = std::max(X->nPmax, pofs[last] - pofs[c] + 1);
    }
    // (dnI, window) work list: windows of TN frequencies with a non-empty n1 range,
    // those whose w window starts at an even column (dn even, since a and m0 are
    // multiples of 2) first
    std::vector<int2> work, work_odd;
    const int nwin = (d.Nw2 + TN - 1) / TN;
    for (int dnI = 0; dnI < d.ndn; ++dnI) {
        const int dn = dnI - (d.Nw2 - 1);
        for (int w = 0; w < nwin; ++w) {
            const int a = w * TN;
            const int lo = std::max(a, std::max(0, -dn)), hi = std::min(a + TN, std::min(d.Nw2, d.Nw2 - dn));
            if (lo < hi) ((dn & 1) ? work_odd : work).push_back(make_int2(dnI, w));
        }
    }
    X->nwork_even = (int)work.size();
    work.insert(work.end(), work_odd.begin(), work_odd.end());
    X->nwork = (int)work.size();
    cudaError_t e = cudaMalloc((void**)&X->work, work.size() * sizeof(int2));
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "cudaMalloc exchange work list");
    e = cudaMemcpy(X->work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange work list upload");

    // stage sizes: JC batch entries per stage; three stages per block, with as
    // many blocks per SM as the register count allows sharing the 227 KB
    cudaFuncAttributes fa;
    cudaError_t fe;
    if (MW == 8) fe = cudaFuncGetAttributes(&fa, k_exchange<4, 8, 0, kSame>);
    else if (MW == 4) fe = cudaFuncGetAttributes(&fa, k_exchange<8, 4, 0, kSame>);
    else if (MW == 2) fe = cudaFuncGetAttributes(&fa, k_exchange<16, 2, 0, kSame>);
    else fe = cudaFuncGetAttributes(&fa, k_exchange<32, 1, 0, kSame>);
    if (fe != cudaSuccess) return g4_cuda_fail(h, fe, "exchange attributes");
    const int regs = fa.numRegs > 0 ? fa.numRegs : 128;
    int per_sm = 65536 / (((regs + 7) / 8 * 8) * X->chunk);
    per_sm = std::max(1, std::min(per_sm, 4));
    const size_t budget = (size_t)(226 * 1024) / per_sm - 2048;
    const int UW = TN + 2, WW = (TN + MW + 1) & ~1;
    int JC = 16;
    auto bytes_for = [&](int jc) {
        const int u = align128(jc * d.Nc * UW * 8);
        const int w = align128(jc * WW * 8);
        return std::make_pair(u, w);
    };
    while (JC > 2) {
        auto uw = bytes_for(JC);
        if ((size_t)kRing * (uw.first + X->nPmax * uw.second) <= budget) break;
        JC /= 2;
    }
    auto uw = bytes_for(JC);
    X->JC = JC;
    X->uBytes = uw.first;
    X->wBytes = uw.second;
    {
        // the epilogue reuses the ring for [chunk][TN][MW] float2 sums + [chunk] row offsets
        const size_t park = (size_t)X->chunk * (TN * MW + 1) * 8 + 16 + (size_t)X->chunk * 8;
        size_t ringB = (size_t)kRing * (X->uBytes + X->nPmax * X->wBytes);
        if (ringB < park) {
            X->uBytes += (int)((park - ringB + kRing * 128 - 1) / (kRing * 128) * 128);
            ringB = (size_t)kRing * (X->uBytes + X->nPmax * X->wBytes);
        }
        X->smem = ringB + 2 * kRing * sizeof(uint64_t) + (size_t)X->nPmax * sizeof(int);
    }
    if (X->smem > (size_t)kMaxSmem)
        return g4_fail(h, G4_ERR_INVALID, "exchange staging does not fit in shared memory");

    // tensor maps over the diagonal-major G~: (n, k, dnI, dk, j), complex64 elements
    auto enc = get_encoder();
    if (!enc) return g4_fail(h, G4_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    const cuuint64_t dims[5] = {(cuuint64_t)d.Nw2, (cuuint64_t)d.Nc, (cuuint64_t)d.ndn,
                                (cuuint64_t)d.Nc, (cuuint64_t)2 * h->batch};
    const cuuint64_t s1 = (cuuint64_t)d.Nw2 * 8;
    const cuuint64_t strides[4] = {s1, s1 * d.Nc, s1 * d.Nc * d.ndn, s1 * d.Nc * d.ndn * d.Nc};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const cuuint32_t boxU[5] = {(cuuint32_t)UW, (cuuint32_t)d.Nc, 1, 1, (cuuint32_t)JC};
    CUresult r = enc(&X->tmU, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, h->Gd, dims, strides, boxU, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return g4_fail(h, G4_ERR_CUDA, "tensor map for the exchange u operand");
    const cuuint32_t boxW[5] = {(cuuint32_t)WW, 1, 1, 1, (cuuint32_t)JC};
    r = enc(&X->tmW, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, h->Gd, dims, strides, boxW, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return g4_fail(h, G4_ERR_CUDA, "tensor map for the exchange w operand");

    if (MW == 8) e = set_smem<4, 8>(X->V);
    else if (MW == 4) e = set_smem<8, 4>(X->V);
    else if (MW == 2) e = set_smem<16, 2>(X->V);
    else e = set_smem<32, 1>(X->V);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange smem attribute");
    return G4_OK;
}

void free_plan(XPlan* X) {
    if (!X) return;
    if (X->work) cudaFree(X->work);
    delete X;
}

g4_status run_plan(g4_ctx* h, const XPlan& X, int staged) {
    const G4Dims& d = h->d;
    XParams P;
    P.pairs = h->pairs;
    P.kadd = h->kadd;
    P.ksub = h->ksub;
    P.work = X.work;
    P.acc = h->acc;
    P.status = h->dstatus;
    P.d = d;
    P.npairs = h->npairs;
    P.nj = 2 * staged;
    P.nmc = (d.Nwex + X.MW - 1) / X.MW;
    P.JC = X.JC;
    P.uBytes = X.uBytes;
    P.wBytes = X.wBytes;
    P.nPmax = X.nPmax;
    P.budget = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : 4000000000LL;
    dim3 grid((h->npairs + X.chunk - 1) / X.chunk, X.nwork, d.Nc * P.nmc);
    if (X.MW == 8) launch<4, 8>(X, P, grid, h->stream);
    else if (X.MW == 4) launch<8, 4>(X, P, grid, h->stream);
    else if (X.MW == 2) launch<16, 2>(X, P, grid, h->stream);
    else launch<32, 1>(X, P, grid, h->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange launch");
    return G4_OK;
}

// ---------------------------------------------------------------- autotuner
// Candidates: every register-tile shape whose m extent does not exceed the
// problem's (MW <= the power of two >= Nwex) times three block sizes.  Each is
// timed (CUDA events, best of two after a warm-up) on the handle's own buffers
// over a full batch; the accumulator is unchanged because the staged G is
// still all zero.  Results are kept per process and, when the environment
// variable G4_TUNE_CACHE names a file, in that file (one "key=MW,chunk" line
// per GPU model and problem shape).

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;

std::string tune_key(const g4_ctx* h) {
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) name = prop.name;
    for (char& c : name)
        if (c == ' ' || c == '=') c = '_';
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|ch%d|Nc%d|Lx%d|Nw2_%d|Nwex%d|Nkex%d|b%d", name.c_str(),
                  h->d.ch, h->d.Nc, h->d.Lx, h->d.Nw2, h->d.Nwex, h->d.Nkex, h->batch);
    return buf;
}

bool tune_lookup(const std::string& key, std::pair<int, int>* out) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
        *out = it->second;
        return true;
    }
    const char* path = std::getenv("G4_TUNE_CACHE");
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        char* eq = std::strchr(line, '=');
        if (!eq) continue;
        *eq = 0;
        int mw = 0, ch = 0;
        if (key == line && std::sscanf(eq + 1, "%d,%d", &mw, &ch) == 2) {
            *out = {mw, ch};
            found = true;
        }
    }
    std::fclose(f);
    if (found) g_tune[key] = *out;
    return found;
}

void tune_store(const std::string& key, std::pair<int, int> v) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = v;
    const char* path = std::getenv("G4_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s=%d,%d\n", key.c_str(), v.first, v.second);
    std::fclose(f);
}

}  // namespace

g4_status exchange_prepare(g4_ctx* h) {
    const G4Dims& d = h->d;
    // (k1, q) pairs sorted by the momentum p of their w row -- k1 (+) q for the
    // shifted band, q (-) k1 for the reflected (particle-particle) one -- then k1
    const bool refl = variant_of(d.ch) == kPP;
    std::vector<int> key((size_t)d.Nc * d.Nc);
    for (int a = 0; a < d.Nc; ++a)
        for (int b = 0; b < d.Nc; ++b) {
            const int ax = a % d.Lx, ay = a / d.Lx, bx = b % d.Lx, by = b / d.Lx;
            key[(size_t)a * d.Nc + b] =
                refl ? (bx - ax + d.Lx) % d.Lx + d.Lx * ((by - ay + d.Ly) % d.Ly)   // b (-) a
                     : (ax + bx) % d.Lx + d.Lx * ((ay + by) % d.Ly);                // a (+) b
        }
    std::vector<int> pairs, pofs;
    for (int p = 0; p < d.Nc; ++p)
        for (int k1 = 0; k1 < d.Nc; ++k1)
            for (int q = 0; q < d.Nkex; ++q)
                if (key[(size_t)k1 * d.Nc + q] == p) {
                    pairs.push_back(k1 | (q << 16));
                    pofs.push_back(p);
                }
    h->npairs = (int)pairs.size();
    cudaError_t e = cudaMalloc((void**)&h->pairs, pairs.size() * sizeof(int));
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "cudaMalloc exchange pairs");
    h->bytes += pairs.size() * sizeof(int);
    e = cudaMemcpy(h->pairs, pairs.data(), pairs.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange pairs upload");

    int mwmax = 1;
    while (mwmax < d.Nwex && mwmax < 8) mwmax *= 2;
    std::pair<int, int> best{mwmax, kMaxThreads};
    // (a custom wait budget is a test setting: tuning runs would give up early)
    if (h->opt.autotune && h->opt.timeout_cycles <= 0) {
        const std::string key = tune_key(h);
        if (!tune_lookup(key, &best)) {
            float best_ms = 1e30f;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
                return g4_fail(h, G4_ERR_CUDA, "autotune events");
            const int chunks[3] = {96, 128, 192};
            g4_status st = G4_OK;
            // m chunks start at multiples of MW; the w-window parity split of the
            // launch assumes those starts are even, so MW = 1 only when Nwex = 1
            const int mwmin = d.Nwex > 1 ? 2 : 1;
            for (int mw = mwmax; mw >= mwmin && mw >= mwmax / 4 && st == G4_OK; mw /= 2) {
                for (int ci = 0; ci < 3 && st == G4_OK; ++ci) {
                    XPlan* X = new (std::nothrow) XPlan();
                    if (!X) {
                        st = g4_fail(h, G4_ERR_OOM, "host allocation of an exchange plan");
                        break;
                    }
                    st = make_plan(h, mw, chunks[ci], pofs, X);
                    float ms = 1e30f;
                    for (int rep = 0; rep < 3 && st == G4_OK; ++rep) {
                        cudaEventRecord(e0, h->stream);
                        st = run_plan(h, *X, h->batch);
                        cudaEventRecord(e1, h->stream);
                        if (st == G4_OK && cudaEventSynchronize(e1) == cudaSuccess) {
                            float t = 0.f;
                            cudaEventElapsedTime(&t, e0, e1);
                            if (rep > 0) ms = std::min(ms, t);
                        }
                    }
                    if (st == G4_OK && ms < best_ms) {
                        best_ms = ms;
                        best = {mw, chunks[ci]};
                    }
                    free_plan(X);
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (st != G4_OK) return st;
            tune_store(key, best);
        }
    }
    XPlan* X = new (std::nothrow) XPlan();
    if (!X) return g4_fail(h, G4_ERR_OOM, "host allocation of the exchange plan");
    h->xplan = X;
    return make_plan(h, best.first, best.second, pofs, X);
}

g4_status exchange_run(g4_ctx* h, int staged) {
    return run_plan(h, *(const XPlan*)h->xplan, staged);
}

void exchange_release(g4_ctx* h) {
    free_plan((XPlan*)h->xplan);
    h->xplan = nullptr;
}
