// Private declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "g4.h"

// Problem sizes.  Index conventions follow g4.h: K = k*Nw2 + n.
struct G4Dims {
    int Nc, Lx, Ly;   // cluster
    int Nw2;          // fermionic frequencies (2*Nw)
    int Nwex, Nkex;   // transfers held by this handle (Nwex: bosonic frequencies m0 .. m0+Nwex-1)
    int m0;           // first bosonic transfer frequency of the handle's slab (0 unless sharded)
    int N;            // Nc*Nw2
    int NQ;           // Nkex*Nwex
    long long E;      // N*N*NQ
    int ndn;          // 2*Nw2-1 frequency differences
    int ch;           // g4_channel
};

// The measurements a deferred handle has staged for its next accumulation:
// each one's M and G0 (device pointers, kept valid by the caller) and its sign
// factor r_s (magnitude and whether it is i times that, see g4_gtilde.cuh).
// Passed to the kernels by value.
constexpr int kMaxBatch = 256;
struct G4Slot {
    const void* M;
    const double2* G0;
    float rs;
    int neg;
};
struct G4SlotTable {
    G4Slot s[kMaxBatch];
};

// Channels with a direct (outer-product) term: the magnetic and density forms.
inline bool has_direct(int ch) { return ch == G4_PH_MAGNETIC || ch == G4_PH_DENSITY; }

// Device words of a handle: the status word, then (mixed path) the batch's
// largest |G~| component, the kept operand scale and the pack's redo flag.
constexpr int kStatusWords = 4;

// Device status word bits (written by kernels whose bounded waits give up).
enum : unsigned { G4_DEV_TIMEOUT = 1u, G4_DEV_BADARG = 2u };

// Waits for progress (data a copy or another role will deliver) use the
// handle's timeout budget; after a block has given up, its waits for work it
// already started itself (copies in flight, issued MMAs), which always
// complete, use this fixed budget (about two seconds at 2 GHz) so that no
// block exits with such work outstanding.
constexpr long long kDrainBudget = 4000000000LL;

// Raise a kernel's dynamic shared-memory limit to the most the device allows
// next to the kernel's static shared memory.  The limit belongs to the kernel
// function (all handles share it), so it is never lowered to one launch's size.
template <typename F>
inline cudaError_t raise_smem_limit(F* fn) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

struct g4_ctx {
    unsigned long long uid = 0;      // process-unique identifier (grouped graph cache)
    G4Dims d{};
    g4_options opt{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int batch = 0;         // slots per batch
    int staged = 0;        // measurements staged in the current batch
    double sign_sum = 0.0;
    long long nmeas = 0;
    bool finalized = false;
    std::vector<double> slot_sign;   // host copy of the staged signs
    std::string err;
    size_t bytes = 0;                // device bytes held

    // tables
    int* kadd = nullptr;   // [Nc][Nc]  momentum addition
    int* ksub = nullptr;   // [Nc][Nc]  ksub[a][b] = a (-) b
    // the accumulator, complex FP64 acc[K1][K2][q][m]: both terms of every
    // measurement (the mixed path adds the direct term once per window of
    // batches, see g4_direct_tc.cu); the exported result is acc / sum_r s_r
    double2* acc = nullptr;
    unsigned* dstatus = nullptr;     // device status word
    unsigned* gmax = nullptr;        // largest |G~| component of the staged batch (FP32 bits),
                                     // for the FP16 operand scale; right after dstatus
    unsigned* gscale = nullptr;      // deferred staging: the largest component whose shift is
                                     // the exchange operands' scale (kept while it stays good)
    unsigned* gredo = nullptr;       // deferred staging: the pack has to run again
    unsigned* hstatus = nullptr;     // pinned host mirror

    // FP64 plain path
    double2* Gfull = nullptr;        // [batch][2][N][N]

    // mixed path
    float2* Gd = nullptr;            // [batch*2][Nc dk][ndn][Nc k][Nw2 n] complex64,
                                     // sqrt(s_r) G (so products of two entries carry s_r);
                                     // not allocated on a deferred handle
    bool deferred = false;           // options.deferred: operands formed from M at accumulation
    G4SlotTable* slots = nullptr;    // deferred: the staged measurements (host)
    int Bp = 0;                      // padded batch (exchange GEMM K per spin)
    int* pairs = nullptr;            // exchange (k1,q) pairs sorted by p = k1 (+) q
    int npairs = 0;
    void* dplan = nullptr;           // direct term: operand window, planes, scratch (mixed path)
    void* xplan = nullptr;           // exchange plan on CUDA cores (tensor maps, work list)
    void* xtc = nullptr;             // exchange plan on tensor cores (operands, work list)
    double2* hstage = nullptr;       // device staging for g4_finalize to host memory (lazy)
    void* nfft = nullptr;            // vertex-configuration transform scratch (lazy)

    // launch timing (g4_profile)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev[G4_K_COUNT];   // start/stop pairs
};

// Bracket a launch with events when profiling is on.
inline void prof_begin(g4_ctx* h, int kind) {
    if (!h->prof_on) return;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return;
    }
    cudaEventRecord(a, h->stream);
    h->prof_ev[kind].push_back(a);
    h->prof_ev[kind].push_back(b);
}
inline void prof_end(g4_ctx* h, int kind) {
    if (!h->prof_on || h->prof_ev[kind].empty()) return;
    cudaEventRecord(h->prof_ev[kind].back(), h->stream);
}

// error helpers (g4_api.cu)
g4_status g4_fail(g4_ctx* h, g4_status st, const std::string& msg);
g4_status g4_cuda_fail(g4_ctx* h, cudaError_t e, const char* what);
#define G4_CUDA(h, call)                                            \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return g4_cuda_fail((h), e_, #call); \
    } while (0)

// device allocation counted against the handle's mem_limit (g4_api.cu)
g4_status g4_dalloc_bytes(g4_ctx* h, void** p, size_t bytes);

// kernels (launch wrappers), each returns cudaGetLastError()
cudaError_t launch_build_G_fp64(const void* M, bool m64, const double2* G0, double2* G,
                                int N, cudaStream_t s);
cudaError_t launch_update_fp64(const double2* G, double sign, double2* acc, const int* kadd,
                               const int* ksub, const G4Dims& d, cudaStream_t s);
// out = acc / S in the exported layout, for the n2 planes [n2_0, n2_0 + n2_cnt):
// plane m of the block is written at out + m * out_plane (E / Nwex for the
// whole array with n2_0 = 0, n2_cnt = 2Nw)
cudaError_t launch_finalize(const double2* acc, bool pair, double inv_s, double2* out,
                            const G4Dims& d, int n2_0, int n2_cnt, long long out_plane,
                            cudaStream_t s);
// one measurement's G~ into its batch slot of Gd, its largest component
// joining *gmax; with Gd_slot == nullptr only the largest component is found
// (a deferred handle's pass)
cudaError_t launch_build_G_diag(const void* M, bool m64, const double2* G0, double sign,
                                float2* Gd_slot, const int* ksub, const G4Dims& d,
                                unsigned* gmax, cudaStream_t s);

// mixed-path exchange (g4_exchange.cu)
struct ExchangePlan;
g4_status exchange_prepare(g4_ctx* h);
g4_status exchange_run(g4_ctx* h, int staged);
void exchange_release(g4_ctx* h);

// mixed-path exchange on tensor cores (g4_exchange_tc.cu)
bool xtc_feasible(const G4Dims& d);
g4_status xtc_prepare(g4_ctx* h);
g4_status xtc_run(g4_ctx* h, int staged);
void xtc_release(g4_ctx* h);

// mixed-path direct term on tensor cores (g4_direct_tc.cu): operands of the
// staged batch into the window (flush_due: the next batch would not fit),
// and the window's GEMM added to the accumulator
g4_status direct_prepare(g4_ctx* h);
g4_status direct_pack(g4_ctx* h, int staged, bool* flush_due);
g4_status direct_flush(g4_ctx* h);
void direct_reset(g4_ctx* h);
int direct_fill(const g4_ctx* h);
int direct_window(const g4_ctx* h);
size_t direct_window_bytes(const g4_ctx* h, int fill);
// the window's operand arrays, maximum word, fill and capacity (deferred
// staging: the exchange pack writes the batch's operands there)
void direct_window_ptrs(const g4_ctx* h, float2** araw, float2** braw, unsigned** wmax, int* fill,
                        int* Bw);
g4_status direct_window_copy(g4_ctx* h, void* host, bool to_host);
g4_status direct_set_fill(g4_ctx* h, int fill);
g4_status direct_window_max(g4_ctx* h, unsigned* bits, bool to_host);
void direct_release(g4_ctx* h);

// vertex configuration -> M (g4_nfft.cu).  Writes M for both spins to Mout, or
// to the handle's scratch when Mout is NULL; *Mres receives the buffer used.
g4_status nfft_run(g4_ctx* h, double beta, int n_up, int n_dn, const double* tau, const int* site,
                   const double* Mtau, void* Mout, const void** Mres);
g4_status nfft_reserve(g4_ctx* h, int nmax);
void nfft_release(g4_ctx* h);
