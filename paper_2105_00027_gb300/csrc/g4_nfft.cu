// The step before the G build (Sec. 2): a walker turns its vertex
// configuration into M_sigma by a non-uniform Fourier transform done as
// matrix products,
//
//   M(K1,K2) = 1/(beta Nc) sum_ij e^{i(w1 tau_i - k1.x_i)} Mtau(i,j) e^{-i(w2 tau_j - k2.x_j)},
//
// K = (k, n), w_n = (2(n-Nw)+1) pi/beta, x_i the lattice site of vertex i.
//
// Factorisation.  The phase of a vertex splits into a time part
// E(w,i) = e^{i w tau_i} and a site part e^{-i k.x_i}; vertices on one site
// share the site part.  With the vertices of each spin grouped by site (a
// stable counting sort), the transform is two grouped products, each
// followed by a discrete Fourier transform over the cluster:
//
//   left   T(k1 w1, j) = sum_r e^{-i k1.r} [ sum_{i at r} E(w1,i) Mtau(i,j) ]
//   right  M(K1; k2 w2) = 1/(beta Nc) sum_r e^{+i k2.r} [ sum_{j at r} T(K1,j) conj E(w2,j) ]
//
// The bracketed sums cost 2Nw n^2 (left) and N 2Nw n (right) products
// instead of the N n^2 and N^2 n of the dense form; the cluster transforms
// run separably (x, then y) in shared memory, N n (Lx+Ly) and N^2 (Lx+Ly).
// The result has the layout g4_compute_G consumes, so the G build follows
// unchanged.  The mixed path computes in FP32 (phases reduced in FP64 first),
// the plain path in FP64.
#include <cmath>
#include <new>
#include <vector>

#include <type_traits>

#include "g4_internal.h"
#include "g4_ptx.cuh"

namespace {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C czero() {
    C z;
    z.x = 0;
    z.y = 0;
    return z;
}

__device__ __forceinline__ float fmac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return __fma_rn(a, b, c); }

// acc += t * v (CONJ: acc += conj(t) * v), two fused multiply-adds per part
template <bool CONJ, typename C> __device__ __forceinline__ void cmac(C& acc, C t, C v) {
    acc.x = fmac(t.x, v.x, acc.x);
    acc.x = fmac(CONJ ? t.y : -t.y, v.y, acc.x);
    acc.y = fmac(t.x, v.y, acc.y);
    acc.y = fmac(CONJ ? -t.y : t.y, v.x, acc.y);
}

// e^{i pi x} for x in [-1, 1]
__device__ __forceinline__ float2 unit_phase(float2*, double x) {
    float s, c;
    sincospif((float)x, &s, &c);
    return make_float2(c, s);
}
__device__ __forceinline__ double2 unit_phase(double2*, double x) {
    double s, c;
    sincospi(x, &s, &c);
    return make_double2(c, s);
}

struct NfftArgs {
    const double* tau;    // [n0 + n1] vertex times, spin 0 first
    const int* site;      // [n0 + n1] vertex sites r = ix + Lx*iy
    const double* Mt;     // spin blocks of Mtau, row-major
    int n[2];             // vertices per spin
    long long mbase[2];   // offset of each spin's Mtau block
    int cap;              // vertex capacity of the scratch arrays
    int Nc, Lx, Ly, Nw, Nw2, N;
    int Nw2p, Np;         // row strides of E and Tm (2Nw and N rounded up to 32)
    double inv_beta;
    int* perm;            // [2][cap]   sorted position -> vertex index
    int* off;             // [2][Nc+1]  first sorted position of each site
    unsigned* status;
};

// Stable counting sort of one spin's vertices by site, one block of 32
// warps per spin.  Warp w owns the vertices [w*seg, (w+1)*seg): it counts
// them per site, the block turns the counts into the first sorted position
// of every (site, warp) pair (sites in order, warps in order within a site),
// and the warp places its vertices from there, lanes with the same site in
// lane order.  Vertices whose site is outside [0, Nc) are left out and flag
// the status word; every later step reads only sorted positions below
// off[Nc].
constexpr int kSortWarps = 32;

__global__ void __launch_bounds__(kSortWarps * 32) k_nfft_sort(NfftArgs a) {
    __shared__ int cnt[kSortWarps][257];   // per (warp, site): count, then next position
    __shared__ int tot[257];
    const int sp = blockIdx.x;
    const int n = sp ? a.n[1] : a.n[0], base = sp ? a.n[0] : 0;
    int* perm = a.perm + (size_t)sp * a.cap;
    int* off = a.off + sp * (a.Nc + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = threadIdx.x; t < kSortWarps * 257; t += blockDim.x) (&cnt[0][0])[t] = 0;
    __syncthreads();
    const int seg = (n + kSortWarps - 1) / kSortWarps;
    const int lo = warp * seg, hi = lo + seg < n ? lo + seg : n;
    const unsigned below = (1u << lane) - 1u;
    bool bad = false;
    for (int c0 = lo; c0 < hi; c0 += 32) {
        const int i = c0 + lane;
        const int r = i < hi ? a.site[base + i] : -1;
        const bool ok = (unsigned)r < (unsigned)a.Nc;
        if (i < hi && !ok) bad = true;
        const unsigned same = __match_any_sync(0xffffffffu, ok ? r : a.Nc + lane);
        if (ok && (same & below) == 0) cnt[warp][r] += __popc(same);
    }
    if (bad) atomicOr(a.status, G4_DEV_BADARG);
    __syncthreads();
    if (threadIdx.x < a.Nc) {
        int t = 0;
        for (int w = 0; w < kSortWarps; ++w) t += cnt[w][threadIdx.x];
        tot[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int r = 0; r < a.Nc; ++r) {
            const int c = tot[r];
            tot[r] = t;
            off[r] = t;
            t += c;
        }
        off[a.Nc] = t;
    }
    __syncthreads();
    if (threadIdx.x < a.Nc) {
        int run = tot[threadIdx.x];
        for (int w = 0; w < kSortWarps; ++w) {
            const int c = cnt[w][threadIdx.x];
            cnt[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int c0 = lo; c0 < hi; c0 += 32) {
        const int i = c0 + lane;
        const int r = i < hi ? a.site[base + i] : -1;
        const bool ok = (unsigned)r < (unsigned)a.Nc;
        const unsigned same = __match_any_sync(0xffffffffu, ok ? r : a.Nc + lane);
        const int rank = __popc(same & below);
        if (ok) perm[cnt[warp][r] + rank] = i;
        __syncwarp();
        if (ok && rank == 0) cnt[warp][r] += __popc(same);
        __syncwarp();
    }
}

// The tables of the products, in sorted order: E[sp][g][w] = e^{i w_n tau}
// of vertex perm[g], and Mr[sp][g][p] = Mtau(perm[g], perm[p]) in the
// working precision (row stride cap, 16-byte aligned rows).  Block row y is
// the spin.
__device__ __forceinline__ float narrow(float*, double v) { return g4ptx::f64_to_f32(v); }
__device__ __forceinline__ double narrow(double*, double v) { return v; }

template <typename C>
__global__ void __launch_bounds__(256) k_nfft_tables(NfftArgs a, C* __restrict__ E,
                                                     decltype(C::x)* __restrict__ Mr) {
    using R = decltype(C::x);
    const int sp = blockIdx.y;
    const int n = sp ? a.n[1] : a.n[0], base = sp ? a.n[0] : 0;
    const int* perm = a.perm + (size_t)sp * a.cap;
    const int ns = a.off[sp * (a.Nc + 1) + a.Nc];
    const double* Mt = a.Mt + (sp ? a.mbase[1] : a.mbase[0]);
    const long long nE = (long long)n * a.Nw2;
    const long long total = nE + (long long)n * n;
    bool bad = false;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < nE) {
            const int g = (int)(e / a.Nw2);
            const int w = (int)(e - (long long)g * a.Nw2);
            if (g >= ns) continue;
            const double t = a.tau[base + perm[g]];
            if (!isfinite(t)) bad = true;
            // w_n tau / pi = (2(n-Nw)+1) tau/beta, reduced exactly to [-1, 1]
            const double x = (double)(2 * (w - a.Nw) + 1) * (t * a.inv_beta);
            const double xr = x - 2.0 * rint(0.5 * x);
            E[((size_t)sp * a.cap + g) * a.Nw2p + w] = unit_phase((C*)nullptr, isfinite(t) ? xr : 0.0);
        } else {
            const long long l = e - nE;
            const int g = (int)(l / n), q = (int)(l - (long long)g * n);
            if (g >= ns || q >= ns) continue;
            Mr[((size_t)sp * a.cap + g) * a.cap + q] =
                narrow((R*)nullptr, Mt[(size_t)perm[g] * n + perm[q]]);
        }
    }
    if (bad) atomicOr(a.status, G4_DEV_BADARG);
}

// Roots of unity of the cluster transforms, e^{-2 pi i m/Lx} then
// e^{-2 pi i m/Ly}, from the FP64 table into shared memory.
template <typename C>
__device__ void load_roots(C* rx, const double2* __restrict__ roots, int Lx, int Ly) {
    for (int m = threadIdx.x; m < Lx + Ly; m += blockDim.x) {
        const double2 v = roots[m];
        rx[m].x = v.x;
        rx[m].y = v.y;
    }
}

// In-place cluster transform of A[r][tile] (r = ix + Lx*iy) over r:
// A[k] = sum_r e^{-+ i k.r} A[r] (CONJ: the + sign), via B.  Separable: x
// then y.  Ends with a barrier.
template <bool CONJ, typename C>
__device__ void cluster_dft(C* A, C* B, const C* rx, const C* ry, int Lx, int Ly, int tile) {
    const int total = Lx * Ly * tile;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int r = e / tile, q = e - r * tile;
        const int kx = r % Lx, iy = r / Lx;
        const C* src = A + (size_t)(Lx * iy) * tile + q;
        C acc = czero<C>();
        int m = 0;
        for (int ix = 0; ix < Lx; ++ix) {
            cmac<CONJ>(acc, rx[m], src[(size_t)ix * tile]);
            m += kx;
            if (m >= Lx) m -= Lx;
        }
        B[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int r = e / tile, q = e - r * tile;
        const int kx = r % Lx, ky = r / Lx;
        const C* src = B + (size_t)kx * tile + q;
        C acc = czero<C>();
        int m = 0;
        for (int iy = 0; iy < Ly; ++iy) {
            cmac<CONJ>(acc, ry[m], src[(size_t)iy * Lx * tile]);
            m += ky;
            if (m >= Ly) m -= Ly;
        }
        A[e] = acc;
    }
    __syncthreads();
}

// Fallback for clusters wider than 8 sites in a direction (the grouped
// kernels below keep their cluster transform in registers).
//
// Left product.  Block (j-block, w-block, spin): for XB sorted vertex
// columns j and WB frequencies w,
//   A[r][j][w] = sum_{sorted g at site r} E(w, g) Mr(g, j),
// then the cluster transform over r gives T(k w, j), stored as
// Tm[sp][j][K = k*2Nw + w] (row stride Np).
template <typename C>
__global__ void __launch_bounds__(256)
k_nfft_left_any(NfftArgs a, const C* __restrict__ E, const decltype(C::x)* __restrict__ Mr,
                const double2* __restrict__ roots, C* __restrict__ Tm, int WB, int XB) {
    using R = decltype(C::x);
    extern __shared__ __align__(16) unsigned char smem[];
    const int tile = WB * XB;
    C* A = (C*)smem;
    C* B = A + (size_t)a.Nc * tile;
    C* rx = B + (size_t)a.Nc * tile;
    C* ry = rx + a.Lx;
    const int sp = blockIdx.z;
    const int* off = a.off + sp * (a.Nc + 1);
    const int ns = off[a.Nc];
    const int p0 = blockIdx.x * XB, w0 = blockIdx.y * WB;
    if (p0 >= ns) return;
    load_roots(rx, roots, a.Lx, a.Ly);
    const R* Ms = Mr + (size_t)sp * a.cap * a.cap;
    const C* Es = E + (size_t)sp * a.cap * a.Nw2p;
    for (int e = threadIdx.x; e < a.Nc * tile; e += blockDim.x) {
        const int r = e / tile, q = e - r * tile;
        const int xb = q / WB, w = q - xb * WB;
        const int wg = w0 + w, j = p0 + xb;
        C acc = czero<C>();
        if (wg < a.Nw2 && j < ns) {
            const int g1 = off[r + 1];
            for (int g = off[r]; g < g1; ++g) {
                const C ev = Es[(size_t)g * a.Nw2p + wg];
                const R m = Ms[(size_t)g * a.cap + j];
                acc.x = fmac(ev.x, m, acc.x);
                acc.y = fmac(ev.y, m, acc.y);
            }
        }
        A[e] = acc;
    }
    __syncthreads();
    cluster_dft<false>(A, B, rx, ry, a.Lx, a.Ly, tile);
    for (int e = threadIdx.x; e < a.Nc * tile; e += blockDim.x) {
        const int k = e / tile, q = e - k * tile;
        const int xb = q / WB, w = q - xb * WB;
        const int wg = w0 + w, j = p0 + xb;
        if (wg < a.Nw2 && j < ns)
            Tm[((size_t)sp * a.cap + j) * a.Np + (size_t)k * a.Nw2 + wg] = A[e];
    }
}

// Right product.  Block (K1-block, w-block, spin): for XB rows K1 and WB
// frequencies w2,
//   A[r][K1][w2] = sum_{sorted g at site r} T(K1, g) conj E(w2, g),
// then the conjugate cluster transform over r and the factor 1/(beta Nc)
// give M(K1; k2 w2), stored row-major [sp][K1][K2].
template <typename C>
__global__ void __launch_bounds__(256)
k_nfft_right_any(NfftArgs a, const C* __restrict__ E, const double2* __restrict__ roots,
                 const C* __restrict__ Tm, C* __restrict__ Mout, int WB, int XB, double scale) {
    using R = decltype(C::x);
    extern __shared__ __align__(16) unsigned char smem[];
    const int tile = WB * XB;
    C* A = (C*)smem;
    C* B = A + (size_t)a.Nc * tile;
    C* rx = B + (size_t)a.Nc * tile;
    C* ry = rx + a.Lx;
    const int sp = blockIdx.z;
    const int* off = a.off + sp * (a.Nc + 1);
    const int K0 = blockIdx.x * XB, w0 = blockIdx.y * WB;
    load_roots(rx, roots, a.Lx, a.Ly);
    const C* Es = E + (size_t)sp * a.cap * a.Nw2p;
    const C* Ts = Tm + (size_t)sp * a.cap * a.Np;
    for (int e = threadIdx.x; e < a.Nc * tile; e += blockDim.x) {
        const int r = e / tile, q = e - r * tile;
        const int xb = q / WB, w = q - xb * WB;
        const int wg = w0 + w, K1 = K0 + xb;
        C acc = czero<C>();
        if (wg < a.Nw2 && K1 < a.N) {
            const int g1 = off[r + 1];
            for (int g = off[r]; g < g1; ++g)
                cmac<true>(acc, Es[(size_t)g * a.Nw2p + wg], Ts[(size_t)g * a.Np + K1]);
        }
        A[e] = acc;
    }
    __syncthreads();
    cluster_dft<true>(A, B, rx, ry, a.Lx, a.Ly, tile);
    const R s = (R)scale;
    for (int e = threadIdx.x; e < a.Nc * tile; e += blockDim.x) {
        const int k = e / tile, q = e - k * tile;
        const int xb = q / WB, w = q - xb * WB;
        const int wg = w0 + w, K1 = K0 + xb;
        if (wg < a.Nw2 && K1 < a.N) {
            C v = A[e];
            v.x *= s;
            v.y *= s;
            Mout[((size_t)sp * a.N + K1) * a.N + (size_t)k * a.Nw2 + wg] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Grouped kernels (clusters up to 8 x 8 sites per direction).
//
// A block owns an RT x CT tile of the output columns of every site r.  Its
// warps (a count chosen per cluster, or by the autotuner) take the sites
// round-robin; a warp walks its site's vertices (sorted positions g: the
// contiguous rows off[r] .. off[r+1]-1 of the sorted tables) in chunks of
// kG, staging the operand rows into a per-warp double buffer with cp.async,
// and each lane accumulates an RB x CB block of the tile in registers.
// After all sites, the cluster transform runs in place on the shared-memory
// tile, one line of <= 8 values per thread at a time, and the tile is
// written out.
//
//   left:  rows = frequencies w (X = E rows), columns = sorted vertices p
//          (Y = Mr rows); out Tm[p][k 2Nw + w]
//   right: rows = K1 (X = Tm rows), columns = frequencies w2 (Y = E rows,
//          conjugated); out M[K1][k2 2Nw + w2] * 1/(beta Nc)

constexpr int kG = 8;          // vertices per staged chunk
constexpr int kMaxWarps = 16;  // warps per block: 8, 12 or 16, chosen per cluster

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(g4ptx::smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Twiddles of the two separable passes, tx[kx*8+ix] = e^{-+2 pi i kx ix/Lx}
// and ty likewise, passed as a kernel parameter so that the unrolled line
// transforms read them as constant operands.
template <typename C>
struct DftTw {
    C x[64];
    C y[64];
};

template <typename C, bool LEFT>
struct GroupTypes {
    using R = decltype(C::x);
    using Y = typename std::conditional<LEFT, R, C>::type;   // staged column operand
};

template <typename C, bool LEFT, int RT, int CT>
__host__ __device__ constexpr size_t group_stage_bytes() {
    return (size_t)kG * (RT * sizeof(C) + CT * sizeof(typename GroupTypes<C, LEFT>::Y));
}

template <typename C, bool LEFT, int RT, int CT>
__host__ __device__ constexpr size_t group_smem_bytes_fixed(int nw) {
    return 2 * (size_t)nw * group_stage_bytes<C, LEFT, RT, CT>() + sizeof(DftTw<C>);
}

// Short transforms of one line held in registers, in place:
// v[k] <- sum_i e^{-+2 pi i k i/L} v[i] (CONJ: the + sign), for L = 2, 3, 4,
// 6 (prime-factor 2 x 3: no twiddles) and 8 (radix 2 over two 4-point
// transforms).
template <typename C> __device__ __forceinline__ C cadd(C a, C b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename C> __device__ __forceinline__ C csub(C a, C b) {
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
// z * e^{-+ i pi/2} = z * (-i) or z * i
template <bool CONJ, typename C> __device__ __forceinline__ C cquarter(C z) {
    C r;
    r.x = CONJ ? -z.y : z.y;
    r.y = CONJ ? z.x : -z.x;
    return r;
}
template <bool CONJ, typename C> __device__ __forceinline__ void fft2(C& a, C& b) {
    const C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}
template <bool CONJ, typename C> __device__ __forceinline__ void fft3(C& a0, C& a1, C& a2) {
    using R = decltype(C::x);
    const R sig = CONJ ? (R)0.86602540378443864676 : (R)-0.86602540378443864676;   // Im e^{-+2 pi i/3}
    const C t = cadd(a1, a2), u = csub(a1, a2);
    C m;
    m.x = fmac((R)-0.5, t.x, a0.x);
    m.y = fmac((R)-0.5, t.y, a0.y);
    C isu;
    isu.x = -sig * u.y;
    isu.y = sig * u.x;
    a0 = cadd(a0, t);
    a1 = cadd(m, isu);
    a2 = csub(m, isu);
}
template <bool CONJ, typename C> __device__ __forceinline__ void fft4(C& v0, C& v1, C& v2, C& v3) {
    const C a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = cquarter<CONJ>(csub(v1, v3));
    v0 = cadd(a, c);
    v1 = cadd(b, d);
    v2 = csub(a, c);
    v3 = csub(b, d);
}
template <bool CONJ, int L, typename C> __device__ __forceinline__ void line_fft(C (&v)[L]) {
    using R = decltype(C::x);
    if constexpr (L == 2) {
        fft2<CONJ>(v[0], v[1]);
    } else if constexpr (L == 3) {
        fft3<CONJ>(v[0], v[1], v[2]);
    } else if constexpr (L == 4) {
        fft4<CONJ>(v[0], v[1], v[2], v[3]);
    } else if constexpr (L == 6) {
        // input n = 3 n1 + 2 n2 (mod 6), output k = 3 k1 + 4 k2 (mod 6)
        C y0 = v[0], y1 = v[2], y2 = v[4], z0 = v[3], z1 = v[5], z2 = v[1];
        fft3<CONJ>(y0, y1, y2);
        fft3<CONJ>(z0, z1, z2);
        v[0] = cadd(y0, z0);
        v[3] = csub(y0, z0);
        v[4] = cadd(y1, z1);
        v[1] = csub(y1, z1);
        v[2] = cadd(y2, z2);
        v[5] = csub(y2, z2);
    } else if constexpr (L == 8) {
        C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        fft4<CONJ>(e0, e1, e2, e3);
        fft4<CONJ>(o0, o1, o2, o3);
        const R h = (R)0.70710678118654752440;   // cos(pi/4)
        C t1, t3;                                  // o1 e^{-+ i pi/4}, o3 e^{-+ 3 i pi/4}
        t1.x = h * (CONJ ? o1.x - o1.y : o1.x + o1.y);
        t1.y = h * (CONJ ? o1.x + o1.y : o1.y - o1.x);
        t3.x = h * (CONJ ? -o3.x - o3.y : o3.y - o3.x);
        t3.y = h * (CONJ ? o3.x - o3.y : -o3.x - o3.y);
        const C t2 = cquarter<CONJ>(o2);
        v[0] = cadd(e0, o0);
        v[4] = csub(e0, o0);
        v[1] = cadd(e1, t1);
        v[5] = csub(e1, t1);
        v[2] = cadd(e2, t2);
        v[6] = csub(e2, t2);
        v[3] = cadd(e3, t3);
        v[7] = csub(e3, t3);
    }
}

template <int L>
constexpr bool kShortFft = L == 2 || L == 3 || L == 4 || L == 6 || L == 8;

// Transform lines of L values at stride st in place: `lines` groups of E
// lines, line (li, e) starting at A + li*lstride + e.  FP32 threads take two
// lines at a time (FP64 one, for registers).  L = 5 and 7 use the twiddle
// table tw[k*8+i] (already carrying the sign), the other lengths the short
// transforms above.
template <int L, bool CONJ, typename C>
__device__ __forceinline__ void dft_lines(C* A, int lines, int E, size_t lstride, size_t st,
                                          const C* tw) {
    constexpr int P = sizeof(C) == 8 ? 2 : 1;
    const int total = lines * E;
    for (int t = threadIdx.x; t < total; t += P * blockDim.x) {
        C* b[P];
        bool ok[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int tp = t + p * blockDim.x;
            ok[p] = tp < total;
            b[p] = ok[p] ? A + (size_t)(tp / E) * lstride + (tp % E) : A + (size_t)(t / E) * lstride + (t % E);
        }
        C v[P][L];
#pragma unroll
        for (int i = 0; i < L; ++i)
#pragma unroll
            for (int p = 0; p < P; ++p) v[p][i] = b[p][i * st];
        if constexpr (kShortFft<L>) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                line_fft<CONJ>(v[p]);
                if (ok[p])
#pragma unroll
                    for (int k = 0; k < L; ++k) b[p][k * st] = v[p][k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < L; ++k) {
                C acc[P];
#pragma unroll
                for (int p = 0; p < P; ++p) acc[p] = czero<C>();
#pragma unroll
                for (int i = 0; i < L; ++i)
#pragma unroll
                    for (int p = 0; p < P; ++p) cmac<false>(acc[p], tw[k * 8 + i], v[p][i]);
#pragma unroll
                for (int p = 0; p < P; ++p)
                    if (ok[p]) b[p][k * st] = acc[p];
            }
        }
    }
}

template <bool CONJ, typename C>
__device__ __forceinline__ void dft_pass(C* A, int lines, int E, size_t lstride, size_t st, int L,
                                         const C* tw) {
    switch (L) {
        case 2: dft_lines<2, CONJ>(A, lines, E, lstride, st, tw); break;
        case 3: dft_lines<3, CONJ>(A, lines, E, lstride, st, tw); break;
        case 4: dft_lines<4, CONJ>(A, lines, E, lstride, st, tw); break;
        case 5: dft_lines<5, CONJ>(A, lines, E, lstride, st, tw); break;
        case 6: dft_lines<6, CONJ>(A, lines, E, lstride, st, tw); break;
        case 7: dft_lines<7, CONJ>(A, lines, E, lstride, st, tw); break;
        case 8: dft_lines<8, CONJ>(A, lines, E, lstride, st, tw); break;
        default: break;   // L = 1: the identity
    }
}

// In-place cluster transform of A[r][E] over r = ix + Lx*iy (Lx, Ly <= 8)
// with the sign e^{-i k.r} (CONJ: e^{+i k.r}); tx, ty are the twiddle tables
// of that sign.  Ends with a barrier.
template <bool CONJ, typename C>
__device__ void dft_inplace(C* A, int E, int Lx, int Ly, const C* tx, const C* ty) {
    dft_pass<CONJ>(A, Ly, E, (size_t)Lx * E, (size_t)E, Lx, tx);
    __syncthreads();
    dft_pass<CONJ>(A, Lx, E, (size_t)E, (size_t)Lx * E, Ly, ty);
    __syncthreads();
}

// n consecutive elements of shared memory into registers, 16 bytes at a time
template <int NV, typename T>
__device__ __forceinline__ void lds_vec(T (&dst)[NV], const T* src) {
    static_assert((NV * sizeof(T)) % 16 == 0 || NV * sizeof(T) < 16, "vector width");
    if constexpr (NV * sizeof(T) >= 16) {
        constexpr int NQ = NV * sizeof(T) / 16;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float4 v = reinterpret_cast<const float4*>(src)[q];
            reinterpret_cast<float4*>(dst)[q] = v;
        }
    } else {
#pragma unroll
        for (int q = 0; q < NV; ++q) dst[q] = src[q];
    }
}

template <typename C, bool LEFT, int RT, int CT, int RB, int CB>
__global__ void __launch_bounds__(kMaxWarps * 32, 1)
k_nfft_group(NfftArgs a, const __grid_constant__ DftTw<C> tw, const C* __restrict__ E,
             const decltype(C::x)* __restrict__ Mr, const C* __restrict__ Tm_in, C* __restrict__ out,
             double scale) {
    using R = typename GroupTypes<C, LEFT>::R;
    using Y = typename GroupTypes<C, LEFT>::Y;
    constexpr int LC = CT / CB, LR = RT / RB;
    static_assert(LR * LC == 32, "one warp covers the tile");
    constexpr int TE = RT * CT;
    constexpr size_t STG = group_stage_bytes<C, LEFT, RT, CT>();
    extern __shared__ __align__(16) unsigned char smem[];
    const int sp = blockIdx.z;
    const int* off = a.off + sp * (a.Nc + 1);
    const int ns = off[a.Nc];                  // sorted vertices (valid sites)
    const int row0 = blockIdx.x * RT, col0 = blockIdx.y * CT;
    if (LEFT && col0 >= ns) return;
    C* A = (C*)smem;                                                // [Nc][TE]
    unsigned char* stage = smem + (size_t)a.Nc * TE * sizeof(C);   // [warp][2][STG]
    const int nw = blockDim.x >> 5;
    // FP32 reads the twiddles as constant operands from the parameter; FP64
    // (whose unrolled loops would hold them in registers) from shared memory
    DftTw<C>* tws = (DftTw<C>*)(stage + 2 * (size_t)nw * STG);
    if constexpr (sizeof(C) == 16)
        for (int t = threadIdx.x; t < 128; t += blockDim.x) (t < 64 ? tws->x[t] : tws->y[t - 64]) = t < 64 ? tw.x[t] : tw.y[t - 64];
    const C* tx = sizeof(C) == 16 ? tws->x : tw.x;
    const C* ty = sizeof(C) == 16 ? tws->y : tw.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lr = lane / LC, lc = lane - (lane / LC) * LC;
    unsigned char* wbuf = stage + (size_t)warp * 2 * STG;
    const R* Ms = Mr + (size_t)sp * a.cap * a.cap;
    const C* Es = E + (size_t)sp * a.cap * a.Nw2p;
    const C* Ts = Tm_in + (size_t)sp * a.cap * a.Np;

    // stage sorted rows g = gs .. gs+m-1 into buffer b: X rows [kG][RT], then
    // Y rows [kG][CT]; every row is 16-byte aligned (padded strides), and the
    // columns past the data read padding or stale values whose outputs are
    // never stored
    auto issue = [&](int b, int gs, int m) {
        unsigned char* base = wbuf + (size_t)b * STG;
        unsigned char* xs = base;
        unsigned char* ys = base + (size_t)kG * RT * sizeof(C);
        constexpr int PX = RT * (int)sizeof(C) / 16;
        constexpr int PY = CT * (int)sizeof(Y) / 16;
#pragma unroll
        for (int q0 = 0; q0 < kG * PX; q0 += 32) {
            const int q = q0 + lane, t = q / PX, pc = q - t * PX;
            if (t < m) {
                const size_t g = (size_t)(gs + t);
                const C* src = LEFT ? Es + g * a.Nw2p + row0 : Ts + g * a.Np + row0;
                cp_async16(xs + (size_t)t * RT * sizeof(C) + 16 * pc, (const unsigned char*)src + 16 * pc);
            }
        }
#pragma unroll
        for (int q0 = 0; q0 < kG * PY; q0 += 32) {
            const int q = q0 + lane, t = q / PY, pc = q - t * PY;
            if (t < m) {
                const size_t g = (size_t)(gs + t);
                const Y* src = LEFT ? (const Y*)(Ms + g * a.cap + col0) : (const Y*)(Es + g * a.Nw2p + col0);
                cp_async16(ys + (size_t)t * CT * sizeof(Y) + 16 * pc, (const unsigned char*)src + 16 * pc);
            }
        }
    };

    for (int r = warp; r < a.Nc; r += nw) {
        const int g0 = off[r], cnt = off[r + 1] - g0;
        C acc[RB][CB];
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int j = 0; j < CB; ++j) acc[i][j] = czero<C>();
        const int nch = (cnt + kG - 1) / kG;
        if (nch > 0) issue(0, g0, cnt < kG ? cnt : kG);
        cp_commit();
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) {
                const int rem = cnt - (c + 1) * kG;
                issue((c + 1) & 1, g0 + (c + 1) * kG, rem < kG ? rem : kG);
            }
            cp_commit();
            cp_wait<1>();
            __syncwarp();
            const unsigned char* base = wbuf + (size_t)(c & 1) * STG;
            const C* xs = (const C*)base;
            const Y* ys = (const Y*)(base + (size_t)kG * RT * sizeof(C));
            const int rem = cnt - c * kG, m = rem < kG ? rem : kG;
            auto step = [&](int t) {
                C xv[RB];
                Y yv[CB];
                lds_vec(xv, xs + t * RT + lr * RB);
                lds_vec(yv, ys + t * CT + lc * CB);
#pragma unroll
                for (int j = 0; j < CB; ++j) {
#pragma unroll
                    for (int i = 0; i < RB; ++i) {
                        if constexpr (LEFT) {
                            acc[i][j].x = fmac(xv[i].x, yv[j], acc[i][j].x);
                            acc[i][j].y = fmac(xv[i].y, yv[j], acc[i][j].y);
                        } else {
                            cmac<true>(acc[i][j], yv[j], xv[i]);
                        }
                    }
                }
            };
            if (m == kG) {
                // full chunk: unrolled, so the loads of later rows issue early
#pragma unroll
                for (int t = 0; t < kG; ++t) step(t);
            } else {
                for (int t = 0; t < m; ++t) step(t);
            }
            __syncwarp();
        }
        cp_wait<0>();
        C* Ar = A + (size_t)r * TE;
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                const int rl = lr * RB + i, cl = lc * CB + j;
                // left tiles are stored column-major (rows w contiguous), right row-major
                Ar[LEFT ? cl * RT + rl : rl * CT + cl] = acc[i][j];
            }
    }
    __syncthreads();
    dft_inplace<!LEFT>(A, TE, a.Lx, a.Ly, tx, ty);
    if (LEFT) {
        for (int e = threadIdx.x; e < a.Nc * TE; e += blockDim.x) {
            const int k = e / TE, q = e - k * TE, cl = q / RT, rl = q - cl * RT;
            const int w = row0 + rl, j = col0 + cl;
            if (w < a.Nw2 && j < ns) out[((size_t)sp * a.cap + j) * a.Np + (size_t)k * a.Nw2 + w] = A[e];
        }
    } else {
        const R s = (R)scale;
        for (int e = threadIdx.x; e < a.Nc * TE; e += blockDim.x) {
            const int k = e / TE, q = e - k * TE, rl = q / CT, cl = q - rl * CT;
            const int K1 = row0 + rl, w2 = col0 + cl;
            if (K1 < a.N && w2 < a.Nw2) {
                C v = A[e];
                v.x *= s;
                v.y *= s;
                out[((size_t)sp * a.N + K1) * a.N + (size_t)k * a.Nw2 + w2] = v;
            }
        }
    }
}

constexpr size_t kTileSmem = 96 * 1024;   // fallback kernels: two blocks per SM

// Fallback tile (WB frequencies x XB columns or rows) whose two cluster-sized
// buffers fit kTileSmem.
void choose_tile(const G4Dims& d, size_t csz, int* WB, int* XB, size_t* smem) {
    int tile = 256;
    while (tile > 8 && 2 * (size_t)d.Nc * tile * csz + (size_t)(d.Lx + d.Ly) * csz > kTileSmem)
        tile /= 2;
    *WB = d.Nw2 < tile ? d.Nw2 : tile;
    *XB = tile / *WB > 0 ? tile / *WB : 1;
    *smem = 2 * (size_t)d.Nc * (*WB) * (*XB) * csz + (size_t)(d.Lx + d.Ly) * csz;
}

constexpr size_t kSmemCap = 232448;   // opt-in shared memory per block

// The grouped kernel's tiles (RT x CT, lane block RB x CB), largest first.
template <typename C, bool LEFT, int RT, int CT, int RB, int CB>
struct GroupCfg {
    static size_t smem(int Nc, int nw) {
        return (size_t)Nc * RT * CT * sizeof(C) + group_smem_bytes_fixed<C, LEFT, RT, CT>(nw);
    }
    // default warps per block: the count in {16, 12, 8} that fits and leaves
    // the fewest idle warp-sites (ties: more warps); 0 if none fits
    static int warps(int Nc) {
        int best = 0;
        double eff = 0.0;
        for (int nw : {16, 12, 8}) {
            if (smem(Nc, nw) > kSmemCap) continue;
            const double e = (double)Nc / (nw * ((Nc + nw - 1) / nw));
            if (e > eff + 1e-9) {
                eff = e;
                best = nw;
            }
        }
        return best;
    }
    static cudaError_t attr() { return raise_smem_limit(k_nfft_group<C, LEFT, RT, CT, RB, CB>); }
    static cudaError_t launch(const G4Dims& d, const NfftArgs& a, int nmax, int nw, const C* E,
                              const decltype(C::x)* Mr, const DftTw<C>& tw, const C* Tm, C* out,
                              double scale, cudaStream_t st) {
        dim3 g;
        if (LEFT)
            g = dim3((unsigned)((d.Nw2 + RT - 1) / RT), (unsigned)((nmax + CT - 1) / CT), 2);
        else
            g = dim3((unsigned)((d.N + RT - 1) / RT), (unsigned)((d.Nw2 + CT - 1) / CT), 2);
        k_nfft_group<C, LEFT, RT, CT, RB, CB><<<g, nw * 32, smem(d.Nc, nw), st>>>(a, tw, E, Mr, Tm,
                                                                                 out, scale);
        return cudaGetLastError();
    }
};

constexpr int kGroupCfgs = 5;

// f(cfg) for the tile configuration with index i (largest tile first)
template <typename C, bool LEFT, typename F>
void with_cfg(int i, F&& f) {
    switch (i) {
        case 0: f(GroupCfg<C, LEFT, 16, 32, 4, 4>()); break;
        case 1: f(GroupCfg<C, LEFT, 16, 16, 4, 2>()); break;
        case 2: f(GroupCfg<C, LEFT, 8, 16, 2, 2>()); break;
        case 3: f(GroupCfg<C, LEFT, 8, 8, 2, 1>()); break;
        default: f(GroupCfg<C, LEFT, 4, 8, 1, 1>()); break;
    }
}

// A tile configuration and warp count of one grouped kernel.
struct GroupChoice {
    int cfg = -1;
    int nw = 0;
};

// Default: the largest tile that fits with its default warp count.
template <typename C, bool LEFT>
GroupChoice default_choice(int Nc) {
    GroupChoice c;
    for (int i = 0; i < kGroupCfgs && c.cfg < 0; ++i)
        with_cfg<C, LEFT>(i, [&](auto cfg) {
            const int nw = decltype(cfg)::warps(Nc);
            if (nw) {
                c.cfg = i;
                c.nw = nw;
            }
        });
    return c;
}

// Candidates for the autotuner: every tile that fits with a warp count in
// {4, 6, 8, 9, 12, 16} that leaves at most a quarter of the warp-sites idle.
template <typename C, bool LEFT>
std::vector<GroupChoice> candidates(int Nc) {
    std::vector<GroupChoice> out;
    for (int i = 0; i < kGroupCfgs; ++i)
        with_cfg<C, LEFT>(i, [&](auto cfg) {
            for (int nw : {4, 6, 8, 9, 12, 16}) {
                if (decltype(cfg)::smem(Nc, nw) > kSmemCap) continue;
                const double e = (double)Nc / (nw * ((Nc + nw - 1) / nw));
                if (e >= 0.75) out.push_back({i, nw});
            }
        });
    return out;
}

bool grouped_ok(const G4Dims& d) { return d.Lx <= 8 && d.Ly <= 8; }

// e^{-2 pi i (k i mod L)/L} (left) or its conjugate (right), k, i < L <= 8
template <typename C>
void group_twiddles(const G4Dims& d, DftTw<C>& tw, bool left) {
    const double pi = 3.14159265358979323846;
    for (int u = 0; u < 128; ++u) {
        const int L = u < 64 ? d.Lx : d.Ly, k = (u & 63) >> 3, i = u & 7;
        C v;
        v.x = 0;
        v.y = 0;
        if (k < L && i < L) {
            const double ph = 2.0 * pi * ((k * i) % L) / L;
            v.x = std::cos(ph);
            v.y = left ? -std::sin(ph) : std::sin(ph);
        }
        (u < 64 ? tw.x[u] : tw.y[u - 64]) = v;
    }
}

struct NfftScratch {
    int cap = 0;
    int* perm = nullptr;
    int* off = nullptr;
    void* E = nullptr;         // [2][cap][Nw2p]  e^{i w tau}, sorted vertex order
    void* Tm = nullptr;        // [2][cap][Np]    left product, row p = sorted vertex p
    void* Mr = nullptr;        // [2][cap][cap]   Mtau, rows and columns sorted, working precision
    void* Mout = nullptr;      // [2][N][N], complex64 (mixed) or complex128 (fp64)
    double2* roots = nullptr;  // [Lx + Ly]
    bool attrs = false;
    size_t grown = 0;          // device bytes of perm, E, Tm and Mr
    GroupChoice left, right;   // grouped-kernel configurations (cfg < 0: not chosen yet)
    bool tuned_left = false, tuned_right = false;
};

template <typename T>
g4_status set_attrs(g4_ctx* h) {
    using C = typename cplx_of<T>::type;
    cudaError_t e = raise_smem_limit(k_nfft_left_any<C>);
    if (e == cudaSuccess) e = raise_smem_limit(k_nfft_right_any<C>);
    if (grouped_ok(h->d))
        for (int i = 0; i < kGroupCfgs && e == cudaSuccess; ++i) {
            with_cfg<C, true>(i, [&](auto cfg) { e = decltype(cfg)::attr(); });
            if (e == cudaSuccess) with_cfg<C, false>(i, [&](auto cfg) { e = decltype(cfg)::attr(); });
        }
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "vertex transform attributes");
    return G4_OK;
}

void free_scratch(NfftScratch* S, bool keep_fixed) {
    void* ptrs[] = {S->perm, S->E, S->Tm, S->Mr};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    S->perm = nullptr;
    S->E = S->Tm = S->Mr = nullptr;
    S->cap = 0;
    if (!keep_fixed) {
        void* fixed[] = {S->off, S->Mout, S->roots};
        for (void* p : fixed)
            if (p) cudaFree(p);
        S->off = nullptr;
        S->Mout = nullptr;
        S->roots = nullptr;
    }
}

int pad32(int x) { return (x + 31) / 32 * 32; }

g4_status ensure(g4_ctx* h, int nmax) {
    const bool f64 = h->opt.precision == G4_PREC_FP64;
    const size_t csz = f64 ? sizeof(double2) : sizeof(float2);
    const G4Dims& d = h->d;
    NfftScratch* S = (NfftScratch*)h->nfft;
    if (!S) {
        S = new (std::nothrow) NfftScratch();
        if (!S) return g4_fail(h, G4_ERR_OOM, "host allocation failed");
        h->nfft = S;
    }
    g4_status st;
    // fixed buffers: each allocated only while its own pointer is null, so a
    // failure part-way (e.g. against mem_limit) leaks nothing and counts
    // nothing twice on the next call
    if (!S->off &&
        (st = g4_dalloc_bytes(h, (void**)&S->off, 2 * (size_t)(d.Nc + 1) * sizeof(int))) != G4_OK)
        return st;
    if (!S->Mout && (st = g4_dalloc_bytes(h, &S->Mout, 2 * (size_t)d.N * d.N * csz)) != G4_OK)
        return st;
    if (!S->roots) {
        if ((st = g4_dalloc_bytes(h, (void**)&S->roots, (size_t)(d.Lx + d.Ly) * sizeof(double2))) != G4_OK)
            return st;
        std::vector<double2> roots((size_t)(d.Lx + d.Ly));
        const double pi = 3.14159265358979323846;
        for (int m = 0; m < d.Lx; ++m)
            roots[m] = make_double2(std::cos(2.0 * pi * m / d.Lx), -std::sin(2.0 * pi * m / d.Lx));
        for (int m = 0; m < d.Ly; ++m)
            roots[d.Lx + m] = make_double2(std::cos(2.0 * pi * m / d.Ly), -std::sin(2.0 * pi * m / d.Ly));
        G4_CUDA(h, cudaMemcpy(S->roots, roots.data(), roots.size() * sizeof(double2),
                              cudaMemcpyHostToDevice));
    }
    if (!S->attrs) {
        if ((st = f64 ? set_attrs<double>(h) : set_attrs<float>(h)) != G4_OK) return st;
        S->attrs = true;
    }
    if (nmax > S->cap) {
        // grow to the next multiple of 256 (the stream is drained first); the
        // bytes of the growable buffers are counted as they are allocated, so
        // a failure part-way leaves the handle's count exact
        G4_CUDA(h, cudaStreamSynchronize(h->stream));
        free_scratch(S, true);
        h->bytes -= S->grown < h->bytes ? S->grown : h->bytes;
        S->grown = 0;
        const int cap = (nmax + 255) / 256 * 256;
        auto grow = [&](void** ptr, size_t bytes) {
            const g4_status r = g4_dalloc_bytes(h, ptr, bytes);
            if (r == G4_OK) S->grown += bytes;
            return r;
        };
        const size_t eb = 2 * (size_t)cap * pad32(d.Nw2) * csz;
        const size_t tb = 2 * (size_t)cap * pad32(d.N) * csz;
        if ((st = grow((void**)&S->perm, 2 * (size_t)cap * sizeof(int))) != G4_OK) return st;
        if ((st = grow(&S->E, eb)) != G4_OK) return st;
        if ((st = grow(&S->Tm, tb)) != G4_OK) return st;
        if ((st = grow(&S->Mr, 2 * (size_t)cap * cap * (csz / 2))) != G4_OK) return st;
        // the padding of both row strides is read by the tiles and stays zero
        G4_CUDA(h, cudaMemset(S->E, 0, eb));
        G4_CUDA(h, cudaMemset(S->Tm, 0, tb));
        S->cap = cap;
    }
    return G4_OK;
}

// Time the candidates on the handle's stream and keep the fastest in *best
// (which holds the default on entry).  The default runs a few times first so
// that the clocks have left idle, then every candidate is timed once per
// round over three interleaved rounds and scored by its fastest round.  The
// candidates differ only in tiling: each output entry is summed in the same
// order, so they write identical results.
template <typename F>
cudaError_t autotune(g4_ctx* h, const std::vector<GroupChoice>& cands, F&& run, GroupChoice* best) {
    if (cands.size() < 2) return cudaSuccess;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    std::vector<float> tmin(cands.size(), 1e30f);
    for (int w = 0; w < 4 && e == cudaSuccess; ++w) e = run(*best);
    for (int round = 0; round < 3 && e == cudaSuccess; ++round)
        for (size_t i = 0; i < cands.size(); ++i) {
            cudaEventRecord(e0, h->stream);
            if ((e = run(cands[i])) != cudaSuccess) break;
            cudaEventRecord(e1, h->stream);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < tmin[i]) tmin[i] = ms;
        }
    if (e == cudaSuccess) {
        size_t bi = 0;
        for (size_t i = 1; i < cands.size(); ++i)
            if (tmin[i] < tmin[bi]) bi = i;
        *best = cands[bi];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

template <typename T>
cudaError_t launch_all(g4_ctx* h, NfftArgs a, void* Mout) {
    using C = typename cplx_of<T>::type;
    const G4Dims& d = h->d;
    NfftScratch* S = (NfftScratch*)h->nfft;
    using R = decltype(C::x);
    k_nfft_sort<<<2, kSortWarps * 32, 0, h->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        const int nm = a.n[0] > a.n[1] ? a.n[0] : a.n[1];
        const long long total = (long long)nm * d.Nw2 + (long long)nm * nm;
        long long nb = (total + 255) / 256;
        if (nb > 152 * 4) nb = 152 * 4;
        if (nb > 0) {
            k_nfft_tables<C><<<dim3((unsigned)nb, 2), 256, 0, h->stream>>>(a, (C*)S->E, (R*)S->Mr);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    const int nmax = a.n[0] > a.n[1] ? a.n[0] : a.n[1];
    const double scale = a.inv_beta / d.Nc;
    const C* E = (const C*)S->E;
    if (grouped_ok(d)) {
        DftTw<C> twl, twr;
        group_twiddles(d, twl, true);
        group_twiddles(d, twr, false);
        if (S->left.cfg < 0) S->left = default_choice<C, true>(d.Nc);
        if (S->right.cfg < 0) S->right = default_choice<C, false>(d.Nc);
        const bool tune = h->opt.autotune && h->opt.timeout_cycles <= 0;
        auto run_left = [&](GroupChoice c) {
            cudaError_t r = cudaSuccess;
            with_cfg<C, true>(c.cfg, [&](auto cfg) {
                r = decltype(cfg)::launch(d, a, nmax, c.nw, E, (const R*)S->Mr, twl, nullptr, (C*)S->Tm,
                                          0.0, h->stream);
            });
            return r;
        };
        auto run_right = [&](GroupChoice c) {
            cudaError_t r = cudaSuccess;
            with_cfg<C, false>(c.cfg, [&](auto cfg) {
                r = decltype(cfg)::launch(d, a, nmax, c.nw, E, (const R*)S->Mr, twr, (const C*)S->Tm,
                                          (C*)Mout, scale, h->stream);
            });
            return r;
        };
        if (S->left.cfg >= 0 && S->right.cfg >= 0) {
            if (nmax > 0) {
                if (tune && !S->tuned_left) {
                    if ((e = autotune(h, candidates<C, true>(d.Nc), run_left, &S->left)) != cudaSuccess)
                        return e;
                    S->tuned_left = true;
                }
                if ((e = run_left(S->left)) != cudaSuccess) return e;
            }
            if (tune && !S->tuned_right) {
                if ((e = autotune(h, candidates<C, false>(d.Nc), run_right, &S->right)) != cudaSuccess)
                    return e;
                S->tuned_right = true;
            }
            return run_right(S->right);
        }
    }
    int WB, XB;
    size_t smem;
    choose_tile(d, sizeof(C), &WB, &XB, &smem);
    const unsigned wblocks = (unsigned)((d.Nw2 + WB - 1) / WB);
    if (nmax > 0) {
        dim3 g((unsigned)((nmax + XB - 1) / XB), wblocks, 2);
        k_nfft_left_any<C><<<g, 256, smem, h->stream>>>(a, E, (const R*)S->Mr, S->roots, (C*)S->Tm, WB,
                                                        XB);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    dim3 g((unsigned)((d.N + XB - 1) / XB), wblocks, 2);
    k_nfft_right_any<C><<<g, 256, smem, h->stream>>>(a, E, S->roots, (const C*)S->Tm, (C*)Mout, WB,
                                                     XB, scale);
    return cudaGetLastError();
}

}  // namespace

g4_status nfft_run(g4_ctx* h, double beta, int n_up, int n_dn, const double* tau, const int* site,
                   const double* Mtau, void* Mout, const void** Mres) {
    if (!(beta > 0.0) || !std::isfinite(beta))
        return g4_fail(h, G4_ERR_INVALID, "beta must be positive and finite");
    if (n_up < 0 || n_dn < 0 || n_up > G4_MAX_VERTICES || n_dn > G4_MAX_VERTICES)
        return g4_fail(h, G4_ERR_INVALID, "vertex count out of range");
    if (n_up + n_dn > 0 && (!tau || !site || !Mtau))
        return g4_fail(h, G4_ERR_INVALID, "tau, site or Mtau is NULL");
    const int nmax = n_up > n_dn ? n_up : n_dn;
    g4_status st = ensure(h, nmax);
    if (st != G4_OK) return st;
    NfftScratch* S = (NfftScratch*)h->nfft;
    const G4Dims& d = h->d;
    NfftArgs a;
    a.tau = tau;
    a.site = site;
    a.Mt = Mtau;
    a.n[0] = n_up;
    a.n[1] = n_dn;
    a.mbase[0] = 0;
    a.mbase[1] = (long long)n_up * n_up;
    a.cap = S->cap > 0 ? S->cap : 1;
    a.Nc = d.Nc;
    a.Lx = d.Lx;
    a.Ly = d.Ly;
    a.Nw = d.Nw2 / 2;
    a.Nw2 = d.Nw2;
    a.N = d.N;
    a.Nw2p = pad32(d.Nw2);
    a.Np = pad32(d.N);
    a.inv_beta = 1.0 / beta;
    a.perm = S->perm;
    a.off = S->off;
    a.status = h->dstatus;
    void* out = Mout ? Mout : S->Mout;
    prof_begin(h, G4_K_NFFT);
    cudaError_t e = h->opt.precision == G4_PREC_FP64 ? launch_all<double>(h, a, out)
                                                     : launch_all<float>(h, a, out);
    prof_end(h, G4_K_NFFT);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "vertex transform launch");
    if (Mres) *Mres = out;
    return G4_OK;
}

g4_status nfft_reserve(g4_ctx* h, int nmax) {
    if (nmax < 0 || nmax > G4_MAX_VERTICES) return g4_fail(h, G4_ERR_INVALID, "vertex count out of range");
    g4_status st = ensure(h, nmax);
    if (st != G4_OK) return st;
    G4_CUDA(h, cudaStreamSynchronize(h->stream));
    return G4_OK;
}

void nfft_release(g4_ctx* h) {
    NfftScratch* S = (NfftScratch*)h->nfft;
    if (!S) return;
    free_scratch(S, false);
    delete S;
    h->nfft = nullptr;
}
