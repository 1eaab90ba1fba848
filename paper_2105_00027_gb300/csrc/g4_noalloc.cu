// Allocation-free entry point: one measurement's plain FP64 update of a
// caller-owned accumulator, with the intermediate G kept in a fixed,
// file-scope device array instead of memory from cudaMalloc.
//
// Who needs it: callers that cannot allocate device memory at the point of
// the update -- for example code whose device memory is owned by another
// allocator that has already reserved the GPU (a framework's caching
// allocator), or a measurement loop that must not pay the implicit device
// synchronisation of cudaMalloc/cudaFree.  Everything this path needs beyond
// the caller's inputs and output lives in g4_noalloc_G below.
//
// The array is shared by every call in the process: calls whose work overlaps
// on the GPU (different streams, or different host threads) race on it.  It
// keeps the last call's contents; each call overwrites all of it that it
// reads, so nothing needs clearing between calls.
#include <cudaTypedefs.h>

#include <mutex>

#include "g4_internal.h"

namespace {

constexpr int kMaxN = G4_NOALLOC_MAX_N;

// Scratch for G of both spins: 2 * 256 * 256 complex128 = 2 MiB per device,
// held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double2 g4_noalloc_G[2 * kMaxN * kMaxN];

// Device address of the array, looked up once per device and context (host
// code must not use the symbol itself: on the host it is only a stand-in).
// The address belongs to the context that was current at the lookup; after
// cudaDeviceReset the device gets a new primary context, so the identifier of
// the current context is kept beside the address and a change triggers a new
// lookup.
std::mutex g_mu;
double2* g_ptr[256] = {};
unsigned long long g_ctx[256] = {};

__device__ __forceinline__ double2 na_cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void k_na_build(const double2* __restrict__ M, const double2* __restrict__ G0,
                           double2* __restrict__ G, int N) {
    const size_t NN = (size_t)N * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < 2 * NN;
         e += (size_t)gridDim.x * blockDim.x) {
        const int sp = (int)(e / NN);
        const size_t ij = e - (size_t)sp * NN;
        const int i = (int)(ij / N), j = (int)(ij - (size_t)i * N);
        const double2 gi = G0[sp * N + i], gj = G0[sp * N + j];
        double2 v = na_cmul(na_cmul(gi, M[e]), gj);
        v.x = -v.x;
        v.y = -v.y;
        if (i == j) {
            v.x += gi.x;
            v.y += gi.y;
        }
        G[e] = v;
    }
}

// acc[m][n2][n1][q][k2][k1] += sign * (a b - exchange), one thread per entry.
__global__ void k_na_update(const double2* __restrict__ G, double sign, double2* __restrict__ acc,
                            int Nc, int Lx, int Nw2, int Nwex, int Nkex) {
    const int N = Nc * Nw2, Ly = Nc / Lx;
    const size_t NN = (size_t)N * N;
    const long long E = (long long)N * N * Nkex * Nwex;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < E;
         o += (long long)gridDim.x * blockDim.x) {
        long long t = o;
        const int k1 = (int)(t % Nc); t /= Nc;
        const int k2 = (int)(t % Nc); t /= Nc;
        const int q = (int)(t % Nkex); t /= Nkex;
        const int n1 = (int)(t % Nw2); t /= Nw2;
        const int n2 = (int)(t % Nw2);
        const int m = (int)(t / Nw2);
        const int qx = q % Lx, qy = q / Lx;
        const int k1q = (k1 % Lx + qx) % Lx + Lx * ((k1 / Lx + qy) % Ly);
        const int k2q = (k2 % Lx + qx) % Lx + Lx * ((k2 / Lx + qy) % Ly);
        const int K1 = k1 * Nw2 + n1, K2 = k2 * Nw2 + n2;
        const bool v1 = n1 + m < Nw2, v2 = n2 + m < Nw2;
        const int K1Q = k1q * Nw2 + n1 + m, K2Q = k2q * Nw2 + n2 + m;
        double2 a = make_double2(0, 0), b = make_double2(0, 0), ex = make_double2(0, 0);
        for (int sp = 0; sp < 2; ++sp) {
            const double2* g = G + sp * NN;
            const double sg = sp ? -1.0 : 1.0;
            if (v1) {
                const double2 u = g[(size_t)K1Q * N + K1];
                a.x += sg * u.x;
                a.y += sg * u.y;
            }
            if (v2) {
                const double2 u = g[(size_t)K2 * N + K2Q];
                b.x += sg * u.x;
                b.y += sg * u.y;
            }
            if (v1 && v2) {
                const double2 u = na_cmul(g[(size_t)K2 * N + K1], g[(size_t)K1Q * N + K2Q]);
                ex.x += u.x;
                ex.y += u.y;
            }
        }
        const double2 ab = na_cmul(a, b);
        double2 r = acc[o];
        r.x += sign * (ab.x - ex.x);
        r.y += sign * (ab.y - ex.y);
        acc[o] = r;
    }
}

// Errors are reported like those of g4_create: message via g4_last_error(NULL).
g4_status na_fail(g4_status st, const std::string& msg) { return g4_fail(nullptr, st, msg); }

// Identifier of the current context (driver cuCtxGetId, reached through the
// runtime's entry-point query so that nothing links against libcuda), or 0
// when it cannot be read.
unsigned long long current_ctx_id() {
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static bool looked = false;
    if (!looked) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_cuCtxGetId_v12000)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (PFN_cuCtxGetCurrent_v4000)p;
        looked = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_id || !get_cur || get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Set-up for the current device: find the device address of the scratch
// array.  Runs inside the first call on each device (and again when that
// device's context has been replaced, e.g. after cudaDeviceReset).
g4_status na_scratch(double2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(G4_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return na_fail(G4_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    // the context identifier is read after the lookup on the first call (the
    // lookup is what brings the runtime's context up), before it afterwards
    if (!g_ptr[dev] || current_ctx_id() != g_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g4_noalloc_G);
        if (e != cudaSuccess || !p)
            return na_fail(G4_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_ptr[dev] = (double2*)p;
        g_ctx[dev] = current_ctx_id();
    }
    *out = g_ptr[dev];
    return G4_OK;
}

}  // namespace

extern "C" g4_status g4_update_noalloc(int Nc, int lx, int Nw, int Nwex, int Nkex, const void* M,
                                       const void* G0, double sign, void* acc, void* stream) {
    if (!M || !G0 || !acc) return na_fail(G4_ERR_INVALID, "M, G0 or acc is NULL");
    // the same limits as g4_create
    if (Nc < 1 || Nc > 256 || Nw < 1 || Nw > 64 || Nwex < 1 || Nwex > 64 || Nkex < 1 || Nkex > Nc)
        return na_fail(G4_ERR_INVALID, "problem sizes out of range");
    int Lx = lx;
    if (Lx == 0) {
        Lx = 1;
        while ((Lx + 1) * (Lx + 1) <= Nc) ++Lx;
        if (Lx * Lx != Nc) return na_fail(G4_ERR_INVALID, "Nc is not square; pass lx");
    }
    if (Lx < 1 || Nc % Lx != 0) return na_fail(G4_ERR_INVALID, "lx does not divide Nc");
    const long long N = (long long)Nc * 2 * Nw;
    if (N > kMaxN)
        return na_fail(G4_ERR_INVALID, "Nc*2*Nw = " + std::to_string(N) +
                                           " exceeds the allocation-free limit of " +
                                           std::to_string(kMaxN));
    double2* G = nullptr;
    g4_status st = na_scratch(&G);
    if (st != G4_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t total = 2 * (size_t)N * N;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_na_build<<<blocks, 256, 0, s>>>((const double2*)M, (const double2*)G0, G, (int)N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(G4_ERR_CUDA, std::string("build launch: ") + cudaGetErrorString(e));
    const long long E = N * N * Nkex * Nwex;
    long long ub = (E + 255) / 256;
    if (ub > 152 * 32) ub = 152 * 32;
    k_na_update<<<(int)ub, 256, 0, s>>>(G, sign, (double2*)acc, Nc, Lx, 2 * Nw, Nwex, Nkex);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(G4_ERR_CUDA, std::string("update launch: ") + cudaGetErrorString(e));
    return G4_OK;
}
