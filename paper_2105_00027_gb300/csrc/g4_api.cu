// C ABI of the G4 library: handle lifecycle, argument checking, batching and
// dispatch to the FP64 plain path or the mixed-precision path.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "g4_gtilde.cuh"
#include "g4_internal.h"

namespace {
thread_local std::string g_create_error;

// Handle identifiers: never reused within a process, so a cached grouped graph
// can name its handles without holding pointers that a later handle might
// occupy.
std::atomic<unsigned long long> g_next_uid{1};

// Executable graphs of g4_accumulate_group, one per group signature: the
// handles (by identifier) in launch order, the number of measurements each had
// staged and how full its direct-term window was (which decides where the
// batch's operands go and whether the window is added).  While a group's
// batches keep that shape the graph is relaunched as it is, and each handle's
// window then advances as it did when the graph was captured; a destroyed
// handle takes its graphs with it.
struct GroupKey {
    unsigned long long uid;
    int staged, fill;
    bool operator==(const GroupKey& o) const {
        return uid == o.uid && staged == o.staged && fill == o.fill;
    }
};
struct GroupGraph {
    std::vector<GroupKey> key;
    std::vector<int> fill_after;
    cudaGraphExec_t exec = nullptr;
};
std::mutex g_graph_mu;
std::vector<GroupGraph> g_graphs;

void drop_graphs_of(unsigned long long uid) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (size_t i = 0; i < g_graphs.size();) {
        bool hit = false;
        for (const auto& kv : g_graphs[i].key) hit = hit || kv.uid == uid;
        if (hit) {
            if (g_graphs[i].exec) cudaGraphExecDestroy(g_graphs[i].exec);
            g_graphs.erase(g_graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

template <typename T>
g4_status dalloc(g4_ctx* h, T** p, size_t count) {
    return g4_dalloc_bytes(h, (void**)p, count * sizeof(T));
}

void prof_clear(g4_ctx* h, int kind) {
    for (cudaEvent_t e : h->prof_ev[kind]) cudaEventDestroy(e);
    h->prof_ev[kind].clear();
}

void free_all(g4_ctx* h) {
    for (int k = 0; k < G4_K_COUNT; ++k) prof_clear(h, k);
    exchange_release(h);
    xtc_release(h);
    nfft_release(h);
    direct_release(h);
    void* ptrs[] = {h->kadd, h->ksub, h->acc, h->dstatus, h->Gfull, h->Gd, h->pairs, h->hstage};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->hstatus) cudaFreeHost(h->hstatus);
    h->kadd = h->ksub = h->pairs = nullptr;
    h->acc = nullptr;
    h->dstatus = h->hstatus = nullptr;
    h->Gfull = nullptr;
    h->Gd = nullptr;
    h->hstage = nullptr;
    delete h->slots;
    h->slots = nullptr;
}

// Lattice tables: kadd[a][b] = a (+) b, ksub[a][b] = a (-) b, componentwise
// modulo the cluster shape.
void lattice_tables(int Lx, int Ly, std::vector<int>& kadd, std::vector<int>& ksub) {
    const int Nc = Lx * Ly;
    kadd.resize((size_t)Nc * Nc);
    ksub.resize((size_t)Nc * Nc);
    for (int a = 0; a < Nc; ++a)
        for (int b = 0; b < Nc; ++b) {
            const int ax = a % Lx, ay = a / Lx, bx = b % Lx, by = b / Lx;
            kadd[(size_t)a * Nc + b] = (ax + bx) % Lx + Lx * ((ay + by) % Ly);
            ksub[(size_t)a * Nc + b] = (ax - bx + Lx) % Lx + Lx * ((ay - by + Ly) % Ly);
        }
}

g4_status check_status(g4_ctx* h) {
    // Only meaningful after a stream synchronisation.
    if (*h->hstatus & G4_DEV_TIMEOUT)
        return g4_fail(h, G4_ERR_TIMEOUT, "a device-side wait exceeded its cycle budget");
    if (*h->hstatus & G4_DEV_BADARG)
        return g4_fail(h, G4_ERR_INVALID, "a kernel rejected its launch arguments");
    return G4_OK;
}

g4_status sync_and_check(g4_ctx* h) {
    G4_CUDA(h, cudaMemcpyAsync(h->hstatus, h->dstatus, sizeof(unsigned), cudaMemcpyDeviceToHost,
                               h->stream));
    G4_CUDA(h, cudaStreamSynchronize(h->stream));
    return check_status(h);
}

g4_status accumulate_fp64(g4_ctx* h) {
    const size_t NN = (size_t)h->d.N * h->d.N;
    for (int r = 0; r < h->staged; ++r) {
        prof_begin(h, G4_K_UPDATE_FP64);
        cudaError_t e = launch_update_fp64(h->Gfull + (size_t)r * 2 * NN, h->slot_sign[r], h->acc,
                                           h->kadd, h->ksub, h->d, h->stream);
        prof_end(h, G4_K_UPDATE_FP64);
        if (e != cudaSuccess) return g4_cuda_fail(h, e, "update_fp64 launch");
    }
    return G4_OK;
}

// Exchange-type term: tensor cores (the kernel records its own launches) or
// CUDA cores.
g4_status exchange_term(g4_ctx* h) {
    if (h->xtc) return xtc_run(h, h->staged);
    prof_begin(h, G4_K_EXCHANGE);
    g4_status st = exchange_run(h, h->staged);
    prof_end(h, G4_K_EXCHANGE);
    return st;
}

// The exchange-type term goes into the accumulator every batch; the direct
// term's operands join the window, whose GEMM is added when the next batch
// would not fit (and at g4_finalize).
g4_status accumulate_mixed(g4_ctx* h) {
    if (!has_direct(h->d.ch)) return exchange_term(h);
    bool flush = false;
    g4_status st;
    if (h->deferred) {
        // the exchange pack writes the direct operands at the window's fill;
        // the window then takes the batch
        if (direct_fill(h) + h->staged > direct_window(h))
            return g4_fail(h, G4_ERR_STATE, "direct-term window overflow");
        if ((st = exchange_term(h)) != G4_OK) return st;
        if ((st = direct_pack(h, h->staged, &flush)) != G4_OK) return st;
    } else {
        if ((st = direct_pack(h, h->staged, &flush)) != G4_OK) return st;
        if ((st = exchange_term(h)) != G4_OK) return st;
    }
    return flush ? direct_flush(h) : G4_OK;
}

g4_status do_accumulate(g4_ctx* h) {
    if (h->staged == 0) return G4_OK;
    g4_status st = h->opt.precision == G4_PREC_FP64 ? accumulate_fp64(h) : accumulate_mixed(h);
    if (st != G4_OK) return st;
    h->staged = 0;
    return G4_OK;
}

// Form one measurement's G into the next batch slot (accumulating a full
// batch first).  m64: M is complex64.
g4_status stage_measurement(g4_ctx* h, const void* M, bool m64, const void* G0, double sign) {
    if (h->staged == h->batch) {
        g4_status st = do_accumulate(h);
        if (st != G4_OK) return st;
    }
    const int slot = h->staged;
    cudaError_t e = cudaSuccess;
    if (h->deferred) {
        // nothing runs now: the accumulation forms the operands (and the
        // batch's largest |G~| component) from M
        const g4gt::SignFactor f = g4gt::sign_factor(sign);
        h->slots->s[slot] = G4Slot{M, (const double2*)G0, f.rs, f.neg ? 1 : 0};
    } else if (h->opt.precision == G4_PREC_FP64) {
        const size_t NN = (size_t)h->d.N * h->d.N;
        prof_begin(h, G4_K_BUILD_G);
        e = launch_build_G_fp64(M, m64, (const double2*)G0, h->Gfull + (size_t)slot * 2 * NN,
                                h->d.N, h->stream);
        prof_end(h, G4_K_BUILD_G);
    } else {
        // the largest |G~| of the batch starts again with its first measurement
        if (slot == 0) e = cudaMemsetAsync(h->gmax, 0, sizeof(unsigned), h->stream);
        const size_t jstride = (size_t)h->d.Nc * h->d.ndn * h->d.Nc * h->d.Nw2;
        prof_begin(h, G4_K_BUILD_G);
        if (e == cudaSuccess)
            e = launch_build_G_diag(M, m64, (const double2*)G0, sign,
                                    h->Gd + (size_t)slot * 2 * jstride, h->ksub, h->d, h->gmax,
                                    h->stream);
        prof_end(h, G4_K_BUILD_G);
    }
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "build_G launch");
    h->slot_sign[slot] = sign;
    h->staged++;
    h->sign_sum += sign;
    h->nmeas++;
    return G4_OK;
}

}  // namespace

g4_status g4_fail(g4_ctx* h, g4_status st, const std::string& msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return st;
}

g4_status g4_cuda_fail(g4_ctx* h, cudaError_t e, const char* what) {
    return g4_fail(h, G4_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

g4_status g4_dalloc_bytes(g4_ctx* h, void** p, size_t bytes) {
 if (h->opt.mem_limit > 0 && (long long)(h->bytes + bytes) > h->opt.mem_limit)
        return g4_fail(h, G4_ERR_OOM, "device allocation of " + std::to_string(bytes) +
                                          " bytes exceeds the configured limit");
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return g4_fail(h, G4_ERR_OOM,
                       "cudaMalloc of " + std::to_string(bytes) + " bytes failed (out of memory)");
    }
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "cudaMalloc");
    h->bytes += bytes;
    return G4_OK;
}


extern "C" {

g4_status g4_options_init(g4_options* opt) {
    if (!opt) return G4_ERR_INVALID;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = G4_PREC_MIXED;
    opt->batch = 64;
    opt->autotune = 1;
    return G4_OK;
}

g4_status g4_create(int Nc, int Nw, int Nwex, int Nkex, g4_channel ch, const g4_options* opt_in,
                    g4_handle* out) {
    if (!out) return g4_fail(nullptr, G4_ERR_INVALID, "out handle pointer is NULL");
    *out = nullptr;
    g4_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        g4_options_init(&opt);
    if (ch != G4_PH_MAGNETIC && ch != G4_PP_UPDOWN && ch != G4_PH_DENSITY && ch != G4_PH_TRANSVERSE)
        return g4_fail(nullptr, G4_ERR_INVALID, "unsupported channel");
    if (Nc < 1 || Nc > 256 || Nw < 1 || Nw > 64 || Nwex < 1 || Nwex > 64 || Nkex < 1 ||
        Nkex > Nc)
        return g4_fail(nullptr, G4_ERR_INVALID, "problem sizes out of range");
    if (opt.precision != G4_PREC_FP64 && opt.precision != G4_PREC_MIXED)
        return g4_fail(nullptr, G4_ERR_INVALID, "unknown precision");
    if (opt.exchange < 0 || opt.exchange > 2)
        return g4_fail(nullptr, G4_ERR_INVALID, "options.exchange must be 0, 1 or 2");
    if (opt.operands != G4_OPERANDS_FP16 && opt.operands != G4_OPERANDS_TF32)
        return g4_fail(nullptr, G4_ERR_INVALID, "options.operands must be FP16 or TF32");
    if (opt.accum != G4_ACCUM_FP64 && opt.accum != G4_ACCUM_F32PAIR)
        return g4_fail(nullptr, G4_ERR_INVALID, "options.accum must be FP64 or F32PAIR");
    if (opt.accum == G4_ACCUM_F32PAIR && (opt.precision != G4_PREC_MIXED || opt.exchange == 1))
        return g4_fail(nullptr, G4_ERR_INVALID,
                       "compensated FP32 pairs need the mixed path with the tensor-core exchange");
    if (opt.deferred != 0 && opt.deferred != 1)
        return g4_fail(nullptr, G4_ERR_INVALID, "options.deferred must be 0 or 1");
    if (opt.deferred && (opt.precision != G4_PREC_MIXED || opt.exchange == 1))
        return g4_fail(nullptr, G4_ERR_INVALID,
                       "deferred staging needs the mixed path with the tensor-core exchange");
    if (opt.direct_batches < 0 || opt.direct_batches > 64)
        return g4_fail(nullptr, G4_ERR_INVALID, "options.direct_batches must be in [0, 64]");
    // a slab of the transfer frequencies (one rank's share of a partitioned G4)
    const int wex_first = opt.wex_count > 0 ? opt.wex_first : 0;
    const int wex_count = opt.wex_count > 0 ? opt.wex_count : Nwex;
    if (opt.wex_first < 0 || opt.wex_count < 0 || wex_first + wex_count > Nwex)
        return g4_fail(nullptr, G4_ERR_INVALID, "options.wex_first/wex_count outside [0, Nwex)");
    if (wex_count != Nwex && opt.precision == G4_PREC_MIXED && opt.exchange == 1)
        return g4_fail(nullptr, G4_ERR_INVALID,
                       "a transfer slab needs the tensor-core exchange (options.exchange 0 or 2)");
    if (opt.batch == 0) opt.batch = 64;
    const int maxb = opt.precision == G4_PREC_FP64 ? 64 : kMaxBatch;
    if (opt.batch < 1 || opt.batch > maxb)
        return g4_fail(nullptr, G4_ERR_INVALID, "batch out of range");
    int Lx = opt.lx;
    if (Lx == 0) {
        Lx = 1;
        while ((Lx + 1) * (Lx + 1) <= Nc) ++Lx;
        if (Lx * Lx != Nc)
            return g4_fail(nullptr, G4_ERR_INVALID, "Nc is not square; set options.lx");
    }
    if (Lx < 1 || Nc % Lx != 0)
        return g4_fail(nullptr, G4_ERR_INVALID, "options.lx does not divide Nc");

    g4_ctx* h = new (std::nothrow) g4_ctx();
    if (!h) return g4_fail(nullptr, G4_ERR_OOM, "host allocation failed");
    h->opt = opt;
    h->uid = g_next_uid.fetch_add(1);
    h->stream = (cudaStream_t)opt.stream;
    h->batch = opt.batch;
    h->deferred = opt.deferred != 0;
    G4Dims& d = h->d;
    d.Nc = Nc;
    d.Lx = Lx;
    d.Ly = Nc / Lx;
    d.Nw2 = 2 * Nw;
    d.Nwex = wex_count;
    d.m0 = wex_first;
    d.Nkex = Nkex;
    d.N = Nc * d.Nw2;
    d.NQ = Nkex * d.Nwex;
    d.E = (long long)d.N * d.N * d.NQ;
    d.ndn = 2 * d.Nw2 - 1;
    d.ch = (int)ch;
    h->slot_sign.assign(h->batch, 0.0);

    auto fail = [&](g4_status st) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return st;
    };
    cudaError_t ce = cudaGetDevice(&h->device);
    if (ce != cudaSuccess) {
        g4_cuda_fail(h, ce, "cudaGetDevice");
        return fail(G4_ERR_CUDA);
    }
    std::vector<int> kadd, ksub;
    lattice_tables(d.Lx, d.Ly, kadd, ksub);
    g4_status st;
    if ((st = dalloc(h, &h->kadd, kadd.size())) != G4_OK) return fail(st);
    if ((st = dalloc(h, &h->ksub, ksub.size())) != G4_OK) return fail(st);
    if ((st = dalloc(h, &h->acc, (size_t)d.E)) != G4_OK) return fail(st);
    if ((st = dalloc(h, &h->dstatus, kStatusWords)) != G4_OK) return fail(st);
    h->gmax = h->dstatus + 1;
    h->gscale = h->dstatus + 2;
    h->gredo = h->dstatus + 3;
    ce = cudaHostAlloc((void**)&h->hstatus, sizeof(unsigned), cudaHostAllocDefault);
    if (ce != cudaSuccess) {
        g4_cuda_fail(h, ce, "cudaHostAlloc");
        return fail(G4_ERR_CUDA);
    }
    *h->hstatus = 0;
    const size_t NN = (size_t)d.N * d.N;
    if (opt.precision == G4_PREC_FP64) {
        if ((st = dalloc(h, &h->Gfull, (size_t)h->batch * 2 * NN)) != G4_OK) return fail(st);
    } else {
        // padded batch: a whole number of operand chunks per spin (64 FP16 or 32 TF32 values)
        const int chunk = opt.operands == G4_OPERANDS_FP16 ? 64 : 32;
        h->Bp = (h->batch + chunk - 1) / chunk * chunk;
        if (h->deferred) {
            h->slots = new (std::nothrow) G4SlotTable();
            if (!h->slots) {
                g4_fail(h, G4_ERR_OOM, "host allocation of the slot table");
                return fail(G4_ERR_OOM);
            }
        } else {
            const size_t gd = (size_t)h->batch * 2 * d.Nc * d.ndn * d.Nc * d.Nw2;
            if ((st = dalloc(h, &h->Gd, gd)) != G4_OK) return fail(st);
            // the out-of-grid half of every diagonal row is never written again
            ce = cudaMemset(h->Gd, 0, gd * sizeof(float2));
            if (ce != cudaSuccess) {
                g4_cuda_fail(h, ce, "cudaMemset staged G");
                return fail(G4_ERR_CUDA);
            }
        }
    }
    ce = cudaMemcpy(h->kadd, kadd.data(), kadd.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess)
        ce = cudaMemcpy(h->ksub, ksub.data(), ksub.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        g4_cuda_fail(h, ce, "table upload");
        return fail(G4_ERR_CUDA);
    }
    if (opt.precision == G4_PREC_MIXED) {
        const bool tc = opt.exchange == 2 || (opt.exchange == 0 && xtc_feasible(d));
        if (!tc && (d.Nwex != Nwex || opt.accum == G4_ACCUM_F32PAIR || h->deferred)) {
            g4_fail(h, G4_ERR_INVALID, "no tensor-core exchange tiling for a transfer slab, "
                                       "an accumulator of FP32 pairs or deferred staging");
            return fail(G4_ERR_INVALID);
        }
        if (tc) {
            if ((st = xtc_prepare(h)) != G4_OK) return fail(st);
        } else if ((st = exchange_prepare(h)) != G4_OK) {
            return fail(st);
        }
        if (has_direct(d.ch) && (st = direct_prepare(h)) != G4_OK) return fail(st);
    }
    if ((st = g4_reset(h)) != G4_OK) return fail(st);
    ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) {
        g4_cuda_fail(h, ce, "create sync");
        return fail(G4_ERR_CUDA);
    }
    *out = h;
    return G4_OK;
}

g4_status g4_reset(g4_handle h) {
    if (!h) return G4_ERR_INVALID;
    G4_CUDA(h, cudaMemsetAsync(h->acc, 0, (size_t)h->d.E * sizeof(double2), h->stream));
    G4_CUDA(h, cudaMemsetAsync(h->dstatus, 0, kStatusWords * sizeof(unsigned), h->stream));
    direct_reset(h);
    h->staged = 0;
    h->sign_sum = 0.0;
    h->nmeas = 0;
    h->finalized = false;
    return G4_OK;
}

g4_status g4_compute_G(g4_handle h, const void* M, const void* G0, double sign) {
    if (!h) return G4_ERR_INVALID;
    if (!M || !G0) return g4_fail(h, G4_ERR_INVALID, "M or G0 is NULL");
    if (h->finalized) return g4_fail(h, G4_ERR_STATE, "g4_compute_G after g4_finalize");
    if (h->deferred && (((uintptr_t)M | (uintptr_t)G0) & 15u) != 0)
        return g4_fail(h, G4_ERR_INVALID, "deferred staging needs M and G0 aligned to 16 bytes");
    return stage_measurement(h, M, h->opt.m_complex64 != 0, G0, sign);
}

g4_status g4_compute_G_vertices(g4_handle h, double beta, int n_up, int n_dn, const double* tau,
                                const int* site, const double* Mtau, const void* G0, double sign) {
    if (!h) return G4_ERR_INVALID;
    if (!G0) return g4_fail(h, G4_ERR_INVALID, "G0 is NULL");
    if (h->finalized) return g4_fail(h, G4_ERR_STATE, "g4_compute_G_vertices after g4_finalize");
    if (h->deferred)
        return g4_fail(h, G4_ERR_INVALID, "vertex staging needs a handle without deferred staging");
    const void* M = nullptr;
    g4_status st = nfft_run(h, beta, n_up, n_dn, tau, site, Mtau, nullptr, &M);
    if (st != G4_OK) return st;
    // the transform's output type: complex128 (FP64 handle), complex64 (mixed)
    return stage_measurement(h, M, h->opt.precision != G4_PREC_FP64, G0, sign);
}

g4_status g4_vertex_M(g4_handle h, double beta, int n_up, int n_dn, const double* tau,
                      const int* site, const double* Mtau, void* M) {
    if (!h) return G4_ERR_INVALID;
    if (!M) return g4_fail(h, G4_ERR_INVALID, "M is NULL");
    g4_status st = nfft_run(h, beta, n_up, n_dn, tau, site, Mtau, M, nullptr);
    if (st != G4_OK) return st;
    return sync_and_check(h);
}

g4_status g4_reserve_vertices(g4_handle h, int n_max) {
    if (!h) return G4_ERR_INVALID;
    return nfft_reserve(h, n_max);
}

g4_status g4_accumulate(g4_handle h) {
    if (!h) return G4_ERR_INVALID;
    if (h->finalized) return g4_fail(h, G4_ERR_STATE, "g4_accumulate after g4_finalize");
    return do_accumulate(h);
}

// Several problems in one launch: every handle's accumulate sequence (pack,
// direct term, exchange) is captured as an independent branch of one CUDA
// graph on the shared stream, so the kernels of small problems run side by
// side instead of one after another.
g4_status g4_accumulate_group(g4_handle* hs, int n) {
    if (!hs || n < 1) return G4_ERR_INVALID;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return G4_ERR_INVALID;
        if (hs[i]->opt.precision != G4_PREC_MIXED)
            return g4_fail(hs[i], G4_ERR_INVALID, "group accumulate needs mixed-precision handles");
        if (hs[i]->deferred)
            return g4_fail(hs[i], G4_ERR_INVALID, "group accumulate takes no deferred handle");
        if (hs[i]->stream != hs[0]->stream)
            return g4_fail(hs[i], G4_ERR_INVALID, "group handles must share a stream");
        if (hs[i]->finalized) return g4_fail(hs[i], G4_ERR_STATE, "handle already finalized");
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return g4_fail(hs[i], G4_ERR_INVALID, "handle listed twice");
    }
    std::vector<g4_ctx*> work;
    for (int i = 0; i < n; ++i)
        if (hs[i]->staged > 0) work.push_back(hs[i]);
    if (work.empty()) return G4_OK;
    if (work.size() == 1) return do_accumulate(work[0]);

    g4_ctx* h0 = hs[0];
    const cudaStream_t main = h0->stream;  // may be the legacy stream, which cannot capture
    const int nb = (int)work.size();
    std::vector<GroupKey> key;
    for (g4_ctx* h : work) key.push_back(GroupKey{h->uid, h->staged, direct_fill(h)});
    {
        // a group shape seen before: relaunch its graph
        std::lock_guard<std::mutex> lock(g_graph_mu);
        for (const GroupGraph& gg : g_graphs)
            if (gg.key == key) {
                cudaError_t e = cudaGraphLaunch(gg.exec, main);
                if (e != cudaSuccess) return g4_cuda_fail(h0, e, "grouped accumulate graph launch");
                for (size_t i = 0; i < work.size(); ++i) {
                    work[i]->staged = 0;
                    direct_set_fill(work[i], gg.fill_after[i]);
                }
                return G4_OK;
            }
    }
    std::vector<cudaStream_t> side(nb, nullptr);
    std::vector<cudaEvent_t> joined(nb, nullptr);
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    g4_status st = G4_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&joined[i], cudaEventDisableTiming);
    }
    bool capturing = false;
    if (e == cudaSuccess) {
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        capturing = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaEventRecord(fork, cap);
    for (int i = 0; i < nb && e == cudaSuccess && st == G4_OK; ++i) {
        g4_ctx* h = work[i];
        e = cudaStreamWaitEvent(side[i], fork, 0);
        if (e != cudaSuccess) break;
        const bool prof = h->prof_on;
        h->prof_on = false;  // no timing events inside the graph
        h->stream = side[i];
        st = do_accumulate(h);
        h->stream = main;
        h->prof_on = prof;
        if (st != G4_OK) break;
        e = cudaEventRecord(joined[i], side[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, joined[i], 0);
    }
    if (capturing) {
        cudaError_t ee = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = ee;
    }
    // the graph runs on the handles' stream, ordered after the staged G builds
    if (e == cudaSuccess && st == G4_OK) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess && st == G4_OK) e = cudaGraphLaunch(exec, main);
    if (e == cudaSuccess && st == G4_OK && exec) {
        // kept for the next batches of the same shape (released with its handles)
        std::lock_guard<std::mutex> lock(g_graph_mu);
        GroupGraph gg;
        gg.key = key;
        for (g4_ctx* h : work) gg.fill_after.push_back(direct_fill(h));
        gg.exec = exec;
        g_graphs.push_back(gg);
        exec = nullptr;
    }
    // streams, events and the graph description are released once their work completes
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (int i = 0; i < nb; ++i) {
        if (joined[i]) cudaEventDestroy(joined[i]);
        if (side[i]) cudaStreamDestroy(side[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    if (st != G4_OK) return st;
    if (e != cudaSuccess) return g4_cuda_fail(h0, e, "grouped accumulate graph");
    return G4_OK;
}

g4_status g4_finalize(g4_handle h, void* out, double* sign_sum) {
    if (!h) return G4_ERR_INVALID;
    if (!out) return g4_fail(h, G4_ERR_INVALID, "out is NULL");
    if (h->finalized) return g4_fail(h, G4_ERR_STATE, "g4_finalize called twice");
    g4_status st = do_accumulate(h);
    if (st != G4_OK) return st;
    if ((st = direct_flush(h)) != G4_OK) return st;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    const bool on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
    const double S = h->sign_sum;
    const double inv = S != 0.0 ? 1.0 / S : 1.0;
    const G4Dims& d = h->d;
    const bool pair = h->opt.accum == G4_ACCUM_F32PAIR;
    const long long plane = d.E / d.Nwex;                     // one m plane of the export
    const long long n2_plane = plane / d.Nw2;                 // one (m, n2) block
    if (on_device) {
        prof_begin(h, G4_K_FINALIZE);
        e = launch_finalize(h->acc, pair, inv, (double2*)out, d, 0, d.Nw2, plane, h->stream);
        prof_end(h, G4_K_FINALIZE);
        if (e != cudaSuccess) return g4_cuda_fail(h, e, "finalize launch");
    } else {
        // host output: blocks of a few n2 planes (every m) through a device
        // staging buffer of about 1 GB, kept by the handle after the first use;
        // each block goes to the host as Nwex rows of one 2-D copy
        int cnt = (int)std::max<long long>(1, (1LL << 30) / (n2_plane * d.Nwex * 16));
        cnt = std::min(cnt, d.Nw2);
        const size_t stage = (size_t)cnt * n2_plane * d.Nwex;
        if (!h->hstage && (st = dalloc(h, &h->hstage, stage)) != G4_OK) return st;
        for (int n2 = 0; n2 < d.Nw2 && e == cudaSuccess; n2 += cnt) {
            const int c = std::min(cnt, d.Nw2 - n2);
            prof_begin(h, G4_K_FINALIZE);
            e = launch_finalize(h->acc, pair, inv, h->hstage, d, n2, c, (long long)c * n2_plane,
                                h->stream);
            prof_end(h, G4_K_FINALIZE);
            const size_t w = (size_t)c * n2_plane * sizeof(double2);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync((char*)out + (size_t)n2 * n2_plane * sizeof(double2),
                                      (size_t)plane * sizeof(double2), h->hstage, w, w, d.Nwex,
                                      cudaMemcpyDeviceToHost, h->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return g4_cuda_fail(h, e, "finalize to host");
    }
    if ((st = sync_and_check(h)) != G4_OK) return st;
    h->finalized = true;
    if (sign_sum) *sign_sum = S;
    if (S == 0.0) return g4_fail(h, G4_ERR_ZERO_SIGN, "sum of signs is zero; output unnormalised");
    return G4_OK;
}

g4_status g4_query(g4_handle h, long long* entries, long long* measurements) {
    if (!h) return G4_ERR_INVALID;
    if (entries) *entries = h->d.E;
    if (measurements) *measurements = h->nmeas;
    return G4_OK;
}

namespace {
// Checkpoint file: this header, the FP64 accumulator (E complex128, internal
// layout), then the direct-term window's filled part (both operand arrays,
// [NQ][N][window_fill] complex64 each), so that a restored run continues
// exactly as the interrupted one would have.
struct CkptHeader {
    char magic[8];
    int version, Nc, Lx, Nw2, Nwex, Nkex, precision, channel;
    double sign_sum;
    long long nmeas, E;
    int window_fill, m0;
    unsigned window_max;
    int accum;
    unsigned gscale;   // the kept exchange operand scale (deferred staging), so that a
                       // restored run continues bit for bit
};
constexpr size_t kIoChunk = (size_t)256 << 20;
}  // namespace

g4_status g4_checkpoint(g4_handle h, const char* path) {
    if (!h || !path) return G4_ERR_INVALID;
    g4_status st = do_accumulate(h);
    if (st != G4_OK) return st;
    if ((st = sync_and_check(h)) != G4_OK) return st;
    const size_t one = (size_t)h->d.E * sizeof(double2);
    const int fill = direct_fill(h);
    const size_t wbytes = direct_window_bytes(h, fill);
    std::vector<char> buf, wbuf;
    try {
        buf.resize(std::min(one, kIoChunk));
        wbuf.resize(wbytes);
    } catch (...) {
        return g4_fail(h, G4_ERR_OOM, "host buffer for checkpoint");
    }
    if ((st = direct_window_copy(h, wbuf.data(), true)) != G4_OK) return st;
    unsigned wmax = 0;
    if ((st = direct_window_max(h, &wmax, true)) != G4_OK) return st;
    unsigned gscale = 0;
    G4_CUDA(h, cudaMemcpy(&gscale, h->gscale, sizeof(unsigned), cudaMemcpyDeviceToHost));
    CkptHeader hd{};
    std::memcpy(hd.magic, "G4CKPT4", 8);
    hd.version = 4;
    hd.Nc = h->d.Nc;
    hd.Lx = h->d.Lx;
    hd.Nw2 = h->d.Nw2;
    hd.Nwex = h->d.Nwex;
    hd.Nkex = h->d.Nkex;
    hd.precision = h->opt.precision;
    hd.channel = h->d.ch;
    hd.sign_sum = h->sign_sum;
    hd.nmeas = h->nmeas;
    hd.E = h->d.E;
    hd.window_fill = fill;
    hd.m0 = h->d.m0;
    hd.window_max = wmax;
    hd.accum = h->opt.accum;
    hd.gscale = gscale;
    FILE* f = std::fopen(path, "wb");
    if (!f) return g4_fail(h, G4_ERR_INVALID, std::string("cannot open ") + path);
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
    cudaError_t e = cudaSuccess;
    for (size_t off = 0; ok && off < one; off += kIoChunk) {
        const size_t n = std::min(kIoChunk, one - off);
        e = cudaMemcpy(buf.data(), (const char*)h->acc + off, n, cudaMemcpyDeviceToHost);
        ok = e == cudaSuccess && std::fwrite(buf.data(), 1, n, f) == n;
    }
    ok = ok && (wbytes == 0 || std::fwrite(wbuf.data(), 1, wbytes, f) == wbytes);
    ok = (std::fclose(f) == 0) && ok;
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "checkpoint copy");
    if (!ok) return g4_fail(h, G4_ERR_INVALID, std::string("write failed: ") + path);
    return G4_OK;
}

g4_status g4_restore(g4_handle h, const char* path) {
    if (!h || !path) return G4_ERR_INVALID;
    FILE* f = std::fopen(path, "rb");
    if (!f) return g4_fail(h, G4_ERR_INVALID, std::string("cannot open ") + path);
    CkptHeader hd{};
    if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, "G4CKPT4", 8) != 0) {
        std::fclose(f);
        return g4_fail(h, G4_ERR_INVALID, "not a G4 checkpoint (of this format)");
    }
    if (hd.Nc != h->d.Nc || hd.Lx != h->d.Lx || hd.Nw2 != h->d.Nw2 || hd.Nwex != h->d.Nwex ||
        hd.Nkex != h->d.Nkex || hd.E != h->d.E || hd.precision != h->opt.precision ||
        hd.channel != h->d.ch || hd.m0 != h->d.m0 || hd.accum != h->opt.accum) {
        std::fclose(f);
        return g4_fail(h, G4_ERR_INVALID, "checkpoint is for a different problem");
    }
    if (hd.window_fill < 0 || hd.window_fill > direct_window(h)) {
        std::fclose(f);
        return g4_fail(h, G4_ERR_INVALID, "checkpoint's direct-term window exceeds this handle's");
    }
    const size_t one = (size_t)h->d.E * sizeof(double2);
    const size_t wbytes = direct_window_bytes(h, hd.window_fill);
    std::vector<char> buf, wbuf;
    try {
        buf.resize(std::min(one, kIoChunk));
        wbuf.resize(wbytes);
    } catch (...) {
        std::fclose(f);
        return g4_fail(h, G4_ERR_OOM, "host buffer for restore");
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    bool ok = e == cudaSuccess;
    for (size_t off = 0; ok && off < one; off += kIoChunk) {
        const size_t n = std::min(kIoChunk, one - off);
        ok = std::fread(buf.data(), 1, n, f) == n;
        if (ok) {
            e = cudaMemcpy((char*)h->acc + off, buf.data(), n, cudaMemcpyHostToDevice);
            ok = e == cudaSuccess;
        }
    }
    ok = ok && (wbytes == 0 || std::fread(wbuf.data(), 1, wbytes, f) == wbytes);
    std::fclose(f);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "restore copy");
    if (!ok) return g4_fail(h, G4_ERR_INVALID, "truncated checkpoint");
    g4_status st = direct_set_fill(h, hd.window_fill);
    if (st == G4_OK) st = direct_window_copy(h, wbuf.data(), false);
    if (st == G4_OK) st = direct_window_max(h, &hd.window_max, false);
    if (st != G4_OK) return st;
    G4_CUDA(h, cudaMemcpy(h->gscale, &hd.gscale, sizeof(unsigned), cudaMemcpyHostToDevice));
    h->sign_sum = hd.sign_sum;
    h->nmeas = hd.nmeas;
    h->staged = 0;
    h->finalized = false;
    return G4_OK;
}

g4_status g4_profile(g4_handle h, int enable) {
    if (!h) return G4_ERR_INVALID;
    h->prof_on = enable != 0;
    return G4_OK;
}

g4_status g4_profile_read(g4_handle h, int kind, double* total_ms, long long* launches) {
    if (!h) return G4_ERR_INVALID;
    if (kind < 0 || kind >= G4_K_COUNT) return g4_fail(h, G4_ERR_INVALID, "unknown kernel kind");
    G4_CUDA(h, cudaStreamSynchronize(h->stream));
    double tot = 0.0;
    long long n = 0;
    auto& ev = h->prof_ev[kind];
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) {
            tot += ms;
            ++n;
        } else {
            cudaGetLastError();
        }
    }
    prof_clear(h, kind);
    if (total_ms) *total_ms = tot;
    if (launches) *launches = n;
    return G4_OK;
}

const char* g4_last_error(g4_handle h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

void g4_destroy(g4_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    drop_graphs_of(h->uid);
    free_all(h);
    delete h;
}

g4_status g4_build_G(int N, const void* M, const void* G0, void* G, void* stream) {
    if (N < 1 || !M || !G0 || !G) return g4_fail(nullptr, G4_ERR_INVALID, "bad g4_build_G arguments");
    cudaError_t e = launch_build_G_fp64(M, false, (const double2*)G0, (double2*)G, N,
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return g4_cuda_fail(nullptr, e, "build_G launch");
    return G4_OK;
}

}  // extern "C"
