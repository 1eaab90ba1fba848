/*
 * g4.h -- C ABI of the GB300 library for the G4 measurement step of a DCA
 * quantum Monte Carlo solver (arXiv 2105.00027).
 *
 * What the library computes.  For every measurement r of a run the caller
 * supplies the per-spin configuration matrices M_sigma (N x N) -- or the
 * vertex configuration they are the Fourier transform of (see
 * g4_compute_G_vertices) -- and the bare propagator G0_sigma (a diagonal, N
 * entries).  The library forms
 *
 *     G_sigma(K1,K2) = G0_sigma(K1) d(K1,K2) - G0_sigma(K1) M_sigma(K1,K2) G0_sigma(K2)
 *
 * (the single-particle Green's function each walker hands to its accumulator,
 * Sec. 2), and adds the measurement's sign-weighted two-particle contribution
 *
 *     G4(K1,K2,Q) += s_r [ (sum_s s G_s(K1+Q,K1)) (sum_s' s' G_s'(K2,K2+Q))
 *                          - sum_s G_s(K2,K1) G_s(K1+Q,K2+Q) ]
 *
 * the particle-hole magnetic form of the accumulation written for the
 * particle-particle channel in Eq. (1) (Sec. 2.1).  The first product is the
 * "direct" term, the second the "exchange" term.  At the end G4 is divided by
 * sum_r s_r.  G4 lives on the device for the whole run, as G_t does in Sec. 2;
 * the paper's 1/p partition of G_t across GPUs (Sec. 3.1) becomes, on one GPU,
 * a tiling of G4 over the transfer Q = (q, m).
 *
 * Indices.  Cluster Lx x Ly, Nc = Lx*Ly momenta, k = kx + Lx*ky.  2*Nw
 * fermionic frequencies, n in [0, 2Nw) for w_n = (2(n-Nw)+1) pi/beta.
 * Combined index K = k*2Nw + n, N = Nc*2Nw.  Transfers Q = (q, m) with
 * q in [0,Nkex) a momentum index and m in [0,Nwex) a bosonic frequency;
 * K+Q = (k (+) q, n+m), (+) adding momenta componentwise mod (Lx, Ly).
 * A G entry whose frequency leaves [0, 2Nw) is zero.
 * Spin index 0 is sigma = +1, index 1 is sigma = -1.
 *
 * Exported G4 layout (g4_finalize output): complex128, row-major
 *     [Nwex m][2Nw n2][2Nw n1][Nkex q][Nc k2][Nc k1]
 * i.e. column-major over (k1, k2, q, n1, n2, m).
 *
 * Errors.  Every call returns a g4_status; no C++ exception or abort crosses
 * the ABI.  A handle in an error state keeps its last message for
 * g4_last_error.  Work is enqueued on the handle's stream; a call returns
 * before the GPU has finished unless documented otherwise.
 */
#ifndef G4_H
#define G4_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct g4_ctx* g4_handle;

typedef enum {
    G4_OK = 0,
    G4_ERR_INVALID = 1,    /* bad size, NULL pointer, unsupported option */
    G4_ERR_OOM = 2,        /* device allocation failed (paper: the run crashes, Sec. 4.5) */
    G4_ERR_CUDA = 3,       /* a CUDA call failed; see g4_last_error */
    G4_ERR_STATE = 4,      /* call not allowed in the handle's current state */
    G4_ERR_ZERO_SIGN = 5,  /* sum of signs is zero at g4_finalize */
    G4_ERR_TIMEOUT = 6     /* a bounded device-side wait gave up */
} g4_status;

/* Channels (each Wick's theorem for its correlator, with a spin-diagonal G):
 *   G4_PH_MAGNETIC   s_r [ (sum_s s G_s(K1+Q,K1)) (sum_s' s' G_s'(K2,K2+Q))
 *                          - sum_s G_s(K2,K1) G_s(K1+Q,K2+Q) ]
 *   G4_PP_UPDOWN     s_r sum_s G_s(Q-K2, Q-K1) G_-s(K2, K1)    -- Eq. (1), Sec. 2.1;
 *                    Q-K = (q (-) k, nu_m - w_n), a G entry off the grid is zero
 *   G4_PH_DENSITY    as G4_PH_MAGNETIC without the spin weights s, s'
 *   G4_PH_TRANSVERSE -s_r sum_s G_-s(K2,K1) G_s(K1+Q,K2+Q)
 * The particle-particle and transverse channels have no direct (outer-product)
 * term, so their mixed path runs only the exchange-type kernel. */
typedef enum {
    G4_PH_MAGNETIC = 0,
    G4_PP_UPDOWN = 1,
    G4_PH_DENSITY = 2,
    G4_PH_TRANSVERSE = 3
} g4_channel;

typedef enum {
    G4_PREC_FP64 = 0,      /* plain path: FP64 G, FP64 update per measurement */
    G4_PREC_MIXED = 1      /* batched path: complex64 G, exchange-type term on tensor
                              cores (3-term FP16 or TF32 split, FP32 accumulate) or FP32
                              CUDA cores, added to the FP64 accumulator once per batch;
                              direct term on tensor cores (same split), kept in operand
                              form over a window of batches and added once per window */
} g4_precision;

typedef struct {
    int precision;          /* g4_precision; default G4_PREC_MIXED */
    int batch;              /* measurements staged per g4_accumulate; default 64,
                               max 256 (mixed) / 64 (fp64) */
    int lx;                 /* cluster width Lx; 0 = square (Lx = sqrt(Nc)) */
    int m_complex64;        /* element type of M: 0 = complex128, 1 = complex64 */
    void* stream;           /* cudaStream_t for all work; NULL = legacy default stream */
    long long timeout_cycles; /* bound of every device-side spin wait (clock64 cycles);
                               0 = default (about 2 s) */
    long long mem_limit;    /* refuse device allocations beyond this many bytes
                               (0 = no limit); used to exercise G4_ERR_OOM */
    int autotune;           /* mixed path: 1 (default) times the candidate exchange
                               tilings on the handle's own buffers at g4_create and
                               keeps the fastest (cached per process, and in the file
                               named by the environment variable G4_TUNE_CACHE);
                               0 uses the built-in choice, as does a nonzero
                               timeout_cycles */
    int exchange;           /* mixed path, kernel of the exchange-type term:
                               0 (default) tensor cores when a tiling exists for the
                               sizes (Nwex <= 16), else CUDA cores; 1 CUDA cores
                               (FP32 FMA); 2 tensor cores, G4_ERR_INVALID if no
                               tiling exists */
    int direct_batches;     /* mixed path, channels with a direct term: batches whose
                               direct-term operands (2 Nkex Nwex N complex64 per
                               measurement) are held before their GEMM is added to the
                               accumulator; 0 (default) = as many as fit in 24 GB, at
                               most 8 */
    /* A slab of the transfers: the handle holds only the G4 entries of the
     * bosonic frequencies m = wex_first .. wex_first + wex_count - 1 (all
     * momenta q) -- one rank's share when G4 is partitioned over GPUs (Sec.
     * 3.1).  wex_count = 0 (default): every m.  The handle's exported array is
     * [wex_count][2Nw][2Nw][Nkex][Nc][Nc], the planes m = wex_first .. of the
     * whole problem's export.  The mixed path then needs the tensor-core
     * exchange. */
    int wex_first;
    int wex_count;
    int operands;           /* mixed path, tensor-core operands: G4_OPERANDS_FP16 (default)
                               or G4_OPERANDS_TF32 hi/lo pairs (below) */
    int accum;              /* mixed path with the tensor-core exchange: the running G4
                               sums as G4_ACCUM_FP64 (default; added by asynchronous
                               FP64 reductions performed at L2) or G4_ACCUM_F32PAIR
                               (compensated FP32 pairs hi + lo, 16 bytes per complex
                               entry like FP64, read, added and written back by the
                               kernels) */
    int deferred;           /* mixed path with the tensor-core exchange: 0 (default) forms
                               each measurement's G in g4_compute_G into the handle's batch
                               buffer; 1 defers it: g4_compute_G records M, G0 and the
                               sign and launches nothing, and the accumulation forms the
                               tensor-core operands of the whole batch from M directly,
                               with no intermediate G and no batch buffer (M and G0 must
                               then be 16-byte aligned, else G4_ERR_INVALID; FP16 pairs keep
                               their power-of-two scale from batch to batch while it stays
                               within one binade of the batch's own, and form the batch's
                               operands a second time when it does not).  M and G0 must then
                               stay valid and unchanged until the measurement has been
                               accumulated (its batch is full and the next g4_compute_G
                               enqueues the work, or g4_accumulate, g4_finalize or
                               g4_checkpoint does) and that work has completed on the
                               handle's stream.  g4_compute_G_vertices and
                               g4_accumulate_group return G4_ERR_INVALID on a deferred
                               handle. */
} g4_options;

enum { G4_ACCUM_FP64 = 0, G4_ACCUM_F32PAIR = 1 };

/* Operands of the mixed path's tensor-core GEMMs.  Each complex64 value x
 * becomes a pair hi + lo and every product is hi.hi + hi.lo + lo.hi with FP32
 * accumulation.  FP16 pairs (kind::f16, twice the tensor rate of TF32 and half
 * the operand bytes) carry the same 22 significant bits as TF32 pairs; their
 * narrower exponent range is covered by a power-of-two scale per GEMM, chosen
 * from the largest operand magnitude, that puts the largest value just below
 * 2^14 -- values down to 2^-17 of the largest keep full precision, smaller ones
 * lose it gradually (absolute error below 2^-39 of the largest). */
enum { G4_OPERANDS_FP16 = 0, G4_OPERANDS_TF32 = 1 };

/* Fill *opt with the defaults listed above.  Returns G4_ERR_INVALID on NULL. */
g4_status g4_options_init(g4_options* opt);

/*
 * Create a handle for one G4 problem and allocate its device state (one FP64
 * accumulator of Nc^2 (2Nw)^2 Nkex Nwex complex entries plus staging buffers).
 *   Nc    cluster sites (Nc = Lx*Ly, Lx from opt->lx)       1 <= Nc <= 256
 *   Nw    positive fermionic frequencies (grid of 2*Nw)     1 <= Nw <= 64
 *   Nwex  bosonic transfers m = 0..Nwex-1                   1 <= Nwex <= 64
 *   Nkex  transfer momenta q = 0..Nkex-1                    1 <= Nkex <= Nc
 *   ch    one of g4_channel
 *   opt   options (NULL = defaults); copied, caller keeps ownership
 *   out   receives the handle (NULL on failure)
 * Errors: G4_ERR_INVALID (sizes, channel, options), G4_ERR_OOM, G4_ERR_CUDA.
 */
g4_status g4_create(int Nc, int Nw, int Nwex, int Nkex, g4_channel ch,
                    const g4_options* opt, g4_handle* out);

/*
 * Stage one measurement (Sec. 2: the walker hands G_sigma to the accumulator).
 *   M     device pointer, [2][N][N] row-major complex128 (or complex64 when
 *         opt.m_complex64), spin-major: M_sigma(K1,K2)
 *   G0    device pointer, [2][N] complex128, G0_sigma(K)
 *   sign  the measurement's Monte Carlo sign (any finite double; +-1 in QMC)
 * G is formed on the handle's stream into the next batch slot; M and G0 must
 * stay valid until that work completes (on a handle with options.deferred:
 * until the measurement's batch has been accumulated and that work has
 * completed).  When the batch is full the staged measurements are accumulated
 * first (as by g4_accumulate).
 * Errors: G4_ERR_INVALID (NULL; on a deferred handle also M or G0 not 16-byte
 * aligned), G4_ERR_STATE (after g4_finalize), G4_ERR_CUDA.
 */
g4_status g4_compute_G(g4_handle h, const void* M, const void* G0, double sign);

/*
 * The step before g4_compute_G (Sec. 2: each walker forms its measurement by a
 * non-uniform Fourier transform of its vertex configuration, done as
 * matrix-matrix products).  For each spin the configuration is n_s vertices
 * (time tau_i, lattice site x_i) and the real n_s x n_s matrix Mtau_s; the
 * library forms
 *
 *   M_s(K1,K2) = 1/(beta Nc) sum_ij e^{i(w1 tau_i - k1.x_i)} Mtau_s(i,j) e^{-i(w2 tau_j - k2.x_j)}
 *
 * (w_n = (2(n-Nw)+1) pi/beta, k.x = 2 pi (kx ix / Lx + ky iy / Ly)) and then
 * stages G_s = G0_s d - G0_s M_s G0_s exactly as g4_compute_G does.
 *   beta        inverse temperature, finite and > 0
 *   n_up, n_dn  vertices per spin, 0 <= n <= G4_MAX_VERTICES (0: M_s = 0)
 *   tau         device, double [n_up + n_dn], spin-up vertices first; any
 *               finite value (the phases are 2 beta-periodic)
 *   site        device, int32 [n_up + n_dn], site r = ix + Lx*iy in [0, Nc)
 *   Mtau        device, double [n_up*n_up + n_dn*n_dn], the spin-up block
 *               then the spin-down block, each row-major
 *   G0, sign    as for g4_compute_G
 * The transform runs in FP64 on an FP64 handle and in FP32 (phases reduced in
 * FP64) on a mixed handle.  Work is enqueued on the handle's stream; the
 * inputs must stay valid until it completes.  The first call with more
 * vertices than any earlier call grows the handle's scratch (a device
 * synchronisation and allocation); g4_reserve_vertices does this up front.
 * Errors: G4_ERR_INVALID (NULL with n > 0, beta, counts), G4_ERR_STATE (after
 * g4_finalize), G4_ERR_OOM, G4_ERR_CUDA.  A site outside [0, Nc) or a
 * non-finite tau is detected on the device: that vertex is left out and the
 * next call that synchronises (g4_finalize, g4_checkpoint) returns
 * G4_ERR_INVALID.
 */
#define G4_MAX_VERTICES 16384
g4_status g4_compute_G_vertices(g4_handle h, double beta, int n_up, int n_dn, const double* tau,
                                const int* site, const double* Mtau, const void* G0, double sign);

/*
 * The transform of g4_compute_G_vertices alone, into a caller buffer:
 *   M   device, [2][N][N] row-major, complex128 on an FP64 handle, complex64
 *       on a mixed handle
 * Synchronous: returns after the device has finished, with G4_ERR_INVALID
 * when a site is outside [0, Nc) or a tau is not finite.  Does not stage a
 * measurement.  Other arguments and errors as for g4_compute_G_vertices.
 */
g4_status g4_vertex_M(g4_handle h, double beta, int n_up, int n_dn, const double* tau,
                      const int* site, const double* Mtau, void* M);

/* Grow the vertex scratch for up to n_max vertices per spin now (allocates
 * and synchronises), so later vertex calls allocate nothing.
 * Errors: G4_ERR_INVALID (n_max out of range), G4_ERR_OOM, G4_ERR_CUDA. */
g4_status g4_reserve_vertices(g4_handle h, int n_max);

/*
 * Add every staged measurement to G4 (the updateG4 step of Algorithm 1) and
 * empty the batch.  No-op when nothing is staged.  On a mixed handle the
 * exchange-type term goes into the FP64 accumulator now; the direct term's
 * operands join the handle's window (options.direct_batches), whose GEMM is
 * added when the window is full and at g4_finalize (g4_checkpoint saves the
 * window with the accumulator).
 * Errors: G4_ERR_STATE (after g4_finalize), G4_ERR_CUDA, G4_ERR_TIMEOUT.
 */
g4_status g4_accumulate(g4_handle h);

/*
 * Accumulate the staged batches of n handles in one grouped launch sequence
 * (several independent problems share each kernel launch).  Each handle must
 * be a G4_PREC_MIXED handle on the same stream as hs[0].
 * Errors: as g4_accumulate; G4_ERR_INVALID if a handle does not qualify.
 */
g4_status g4_accumulate_group(g4_handle* hs, int n);

/*
 * Finish the run: accumulate what is staged (and the direct-term window), then
 * write G4 / sum_r s_r in the exported layout.
 *   out       device or host pointer to E = Nc^2 (2Nw)^2 Nkex Nwex complex128;
 *             a host pointer makes the call synchronous, and on its first use
 *             the handle allocates (and keeps) a device staging buffer of about
 *             1 GB through which the result goes to the host in blocks
 *   sign_sum  optional (may be NULL); receives sum_r s_r
 * After this call g4_compute_G and g4_accumulate return G4_ERR_STATE until
 * g4_reset.  If sum_r s_r == 0 the unnormalised sum is written and
 * G4_ERR_ZERO_SIGN is returned.
 */
g4_status g4_finalize(g4_handle h, void* out, double* sign_sum);

/* Zero the accumulator and the sign sum and start a new run. */
g4_status g4_reset(g4_handle h);

/*
 * Save / restore the accumulator state (FP64 sums, the direct-term window's
 * pending operands and scale, the kept exchange operand scale of deferred
 * staging, sign sum, measurement count, problem description) to / from a
 * file.  Staged measurements are accumulated first.  A restored run
 * continues exactly (bit for bit) as the interrupted one would have.
 * Restoring into a handle of a different problem, or one whose direct-term
 * window is smaller than the saved fill, gives G4_ERR_INVALID.  Both calls
 * synchronise the handle's stream.
 */
g4_status g4_checkpoint(g4_handle h, const char* path);
g4_status g4_restore(g4_handle h, const char* path);

/* Query sizes: number of exported entries E and measurements accumulated. */
g4_status g4_query(g4_handle h, long long* entries, long long* measurements);

/*
 * Per-kernel timing with CUDA events recorded on the handle's stream around
 * every launch (for roofline accounting).  Kinds: */
typedef enum {
    G4_K_BUILD_G = 0,      /* G build (either layout) */
    G4_K_PACK = 1,         /* direct-term operands of a batch into the window */
    G4_K_DIRECT = 2,       /* direct-term GEMM of a transfer group (tensor cores) */
    G4_K_EXCHANGE = 3,     /* exchange-type term + FP64 accumulate (either kernel) */
    G4_K_UPDATE_FP64 = 4,  /* plain FP64 per-measurement update */
    G4_K_FINALIZE = 5,     /* normalisation + export transpose */
    G4_K_PACK_EXCHANGE = 6,/* exchange operand pack (tensor-core exchange) */
    G4_K_NFFT = 7,         /* vertex configuration -> M (sort, phases, both products) */
    G4_K_DIRECT_SPLIT = 8, /* direct-term TF32 hi/lo planes of a transfer group */
    G4_K_DIRECT_MERGE = 9, /* direct-term scratch added to the FP64 accumulator */
    G4_K_COUNT = 10
} g4_kernel_kind;

/* enable != 0 starts recording, 0 stops.  Recording adds two event records
 * per launch. */
g4_status g4_profile(g4_handle h, int enable);

/* Synchronise the handle's stream and return, for one kernel kind, the summed
 * device time (ms) and launch count recorded since the last read; the record
 * of that kind is then cleared.  Errors: G4_ERR_INVALID (kind), G4_ERR_CUDA. */
g4_status g4_profile_read(g4_handle h, int kind, double* total_ms, long long* launches);

/* Last error message of the handle (or of the last failed g4_create when h is
 * NULL).  The string stays valid until the next call on the handle. */
const char* g4_last_error(g4_handle h);

/* Free the handle's device state.  NULL is ignored. */
void g4_destroy(g4_handle h);

/*
 * Standalone form of the G build (the step before every update):
 *   G_sigma = G0_sigma d - G0_sigma M_sigma G0_sigma for both spins.
 *   M   device [2][N][N] complex128      G0 device [2][N] complex128
 *   G   device [2][N][N] complex128 (output, row-major)
 *   stream  cudaStream_t or NULL
 * Errors: G4_ERR_INVALID (N < 1 or NULL pointers), G4_ERR_CUDA.
 */
g4_status g4_build_G(int N, const void* M, const void* G0, void* G, void* stream);

/*
 * Allocation-free update (the paper has no counterpart; this exists for
 * callers that cannot allocate device memory when they update G4 -- e.g. code
 * whose GPU memory is owned by another allocator that has already reserved
 * the device, or a measurement loop that must not pay the implicit device
 * synchronisation of cudaMalloc/cudaFree).
 *
 * Adds one measurement's sign-weighted particle-hole magnetic contribution,
 * computed in FP64 as by the G4_PREC_FP64 path, to a caller-owned accumulator:
 *     acc += sign * [direct - exchange]   (no normalisation)
 *   Nc, lx   cluster sites and width (lx = 0: square cluster)
 *   Nw, Nwex, Nkex   as for g4_create
 *   M    device [2][N][N] complex128      G0  device [2][N] complex128
 *   acc  device, E complex128 in the exported layout of g4_finalize; the
 *        caller zeroes it before the first measurement and divides by the
 *        sum of signs at the end
 *   stream  cudaStream_t or NULL
 * The intermediate G of both spins lives in a fixed device array of
 * 2 * G4_NOALLOC_MAX_N^2 complex128 (2 MiB) inside the library, so
 * N = Nc * 2Nw must not exceed G4_NOALLOC_MAX_N (else G4_ERR_INVALID); Nc,
 * Nw, Nwex and Nkex have the limits of g4_create.  The call allocates no
 * memory.  Its first call on each device looks up the array's device address
 * (once, with that device current); make that first call before any stream
 * capture.  The address belongs to the device's context: after
 * cudaDeviceReset the next call looks it up again (treat that call as a first
 * call).  All calls share the array: calls whose work can overlap on the GPU
 * (other streams, other host threads) race on it.  The sizes of M, G0 and acc
 * are not checked by the library (it receives plain pointers).
 * Errors: G4_ERR_INVALID (NULL, sizes), G4_ERR_CUDA; the message is available
 * from g4_last_error(NULL).
 */
#define G4_NOALLOC_MAX_N 256
g4_status g4_update_noalloc(int Nc, int lx, int Nw, int Nwex, int Nkex, const void* M,
                            const void* G0, double sign, void* acc, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* G4_H */
