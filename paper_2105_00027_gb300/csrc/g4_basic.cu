// Element-wise and layout kernels of the G4 path:
//   * G build, G = G0 d - G0 M G0 (Sec. 2), in the natural layout (FP64 path,
//     standalone g4_build_G) and in the diagonal-major complex64 layout the
//     mixed path consumes;
//   * the plain FP64 per-measurement update of the particle-hole magnetic G4
//     (the accumulation of Eq. (1), Sec. 2.1);
//   * the final normalisation by the sign sum and the transpose to the
//     exported layout.
#include <type_traits>

#include "g4_gtilde.cuh"
#include "g4_internal.h"
#include "g4_ptx.cuh"

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <bool M64>
__device__ __forceinline__ double2 load_m(const void* M, size_t i) {
    if (M64) {
        float2 v = reinterpret_cast<const float2*>(M)[i];
        return make_double2(v.x, v.y);
    } else {
        return reinterpret_cast<const double2*>(M)[i];
    }
}

// G[sp][i][j] = G0[sp][i] d_ij - G0[sp][i] M[sp][i][j] G0[sp][j], FP64.
template <bool M64>
__global__ void k_build_G_fp64(const void* __restrict__ M, const double2* __restrict__ G0,
                               double2* __restrict__ G, int N) {
    const size_t NN = (size_t)N * N;
    const size_t total = 2 * NN;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int sp = (int)(e / NN);
        const size_t ij = e - (size_t)sp * NN;
        const int i = (int)(ij / N), j = (int)(ij - (size_t)i * N);
        const double2 gi = G0[sp * N + i], gj = G0[sp * N + j];
        double2 v = cmul(cmul(gi, load_m<M64>(M, e)), gj);
        v.x = -v.x;
        v.y = -v.y;
        if (i == j) {
            v.x += gi.x;
            v.y += gi.y;
        }
        G[e] = v;
    }
}

// One measurement's FP64 update of every accumulator entry, for channel CH
// (see g4.h).  Block row K1 = blockIdx.y; threads run over (K2, Q) with Q
// fastest, so the accumulator read-modify-write is coalesced.
template <int CH>
__global__ void k_update_fp64(const double2* __restrict__ G, double sign,
                              double2* __restrict__ acc, const int* __restrict__ kadd,
                              const int* __restrict__ ksub, G4Dims d) {
    const int K1 = blockIdx.y;
    const int k1 = K1 / d.Nw2, n1 = K1 - k1 * d.Nw2;
    const size_t NN = (size_t)d.N * d.N;
    const int per = d.N * d.NQ;
    double2* row = acc + (size_t)K1 * per;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < per;
         idx += gridDim.x * blockDim.x) {
        const int K2 = idx / d.NQ, Qi = idx - K2 * d.NQ;
        const int q = Qi / d.Nwex, m = d.m0 + Qi - q * d.Nwex;   // m: the transfer frequency
        const int k2 = K2 / d.Nw2, n2 = K2 - k2 * d.Nw2;
        double2 term = make_double2(0, 0);
        if (CH == G4_PP_UPDOWN) {
            // G_s(Q-K2, Q-K1) G_-s(K2, K1); Q-K has frequency index m + Nw2-1 - n
            const int f1 = m + d.Nw2 - 1 - n1, f2 = m + d.Nw2 - 1 - n2;
            if (f1 >= 0 && f1 < d.Nw2 && f2 >= 0 && f2 < d.Nw2) {
                const int QK1 = ksub[q * d.Nc + k1] * d.Nw2 + f1;
                const int QK2 = ksub[q * d.Nc + k2] * d.Nw2 + f2;
#pragma unroll
                for (int sp = 0; sp < 2; ++sp) {
                    const double2 t = cmul(G[sp * NN + (size_t)QK2 * d.N + QK1],
                                           G[(1 - sp) * NN + (size_t)K2 * d.N + K1]);
                    term.x += t.x;
                    term.y += t.y;
                }
            }
        } else {
            const bool v1 = n1 + m < d.Nw2, v2 = n2 + m < d.Nw2;
            const int K1Q = kadd[k1 * d.Nc + q] * d.Nw2 + n1 + m;
            const int K2Q = kadd[k2 * d.Nc + q] * d.Nw2 + n2 + m;
            double2 a = make_double2(0, 0), b = make_double2(0, 0), ex = make_double2(0, 0);
#pragma unroll
            for (int sp = 0; sp < 2; ++sp) {
                const double2* g = G + sp * NN;
                const double wgt = (CH == G4_PH_MAGNETIC && sp) ? -1.0 : 1.0;
                if (CH != G4_PH_TRANSVERSE) {
                    if (v1) {
                        const double2 t = g[(size_t)K1Q * d.N + K1];
                        a.x += wgt * t.x;
                        a.y += wgt * t.y;
                    }
                    if (v2) {
                        const double2 t = g[(size_t)K2 * d.N + K2Q];
                        b.x += wgt * t.x;
                        b.y += wgt * t.y;
                    }
                }
                if (v1 && v2) {
                    // transverse pairs the opposite spin in the G(K2,K1) factor
                    const double2* gx = CH == G4_PH_TRANSVERSE ? G + (1 - sp) * NN : g;
                    const double2 t = cmul(gx[(size_t)K2 * d.N + K1], g[(size_t)K1Q * d.N + K2Q]);
                    ex.x += t.x;
                    ex.y += t.y;
                }
            }
            const double2 ab = cmul(a, b);
            term = make_double2(ab.x - ex.x, ab.y - ex.y);
        }
        double2 o = row[idx];
        o.x += sign * term.x;
        o.y += sign * term.y;
        row[idx] = o;
    }
}

// The same FP64 update for the particle-hole channels, tiled: a block owns a
// momentum pair (k1, k2) and a 16 x 16 tile of frequencies (n1, n2), one thread
// per (n1, n2), and walks the transfer momenta q.  For each q it stages in
// shared memory what the tile's products read -- the window of the G blocks
// (k1 (+) q, k2 (+) q) at rows n1 + m and columns n2 + m (exchange factor), the
// spin-weighted band G(K1+Q, K1) (a) and G(K2, K2+Q) (b) -- next to the fixed
// G(K2, K1) tile, and each thread adds its Nwex transfers m, so that over the
// q walk a thread updates its entries acc[K1][K2][q][m] in order (every line of
// the accumulator written whole).  Nwex <= kTileWex.
constexpr int kTileF = 16;      // frequencies per tile side
constexpr int kTileWex = 16;    // largest Nwex of the tiled form

template <int CH>
__global__ void __launch_bounds__(kTileF * kTileF) k_update_fp64_tiled(
    const double2* __restrict__ G, double sign, double2* __restrict__ acc,
    const int* __restrict__ kadd, G4Dims d) {
    extern __shared__ double2 sm[];
    const int Nw2 = d.Nw2, N = d.N, Nwex = d.Nwex;
    const int nt = (Nw2 + kTileF - 1) / kTileF;
    const int k1 = blockIdx.y / d.Nc, k2 = blockIdx.y - (blockIdx.y / d.Nc) * d.Nc;
    const int n1_0 = (blockIdx.x / nt) * kTileF, n2_0 = (blockIdx.x % nt) * kTileF;
    const int t1 = threadIdx.x / kTileF, t2 = threadIdx.x % kTileF;
    const int n1 = n1_0 + t1, n2 = n2_0 + t2;
    const bool live = n1 < Nw2 && n2 < Nw2;
    const size_t NN = (size_t)N * N;
    const int WX = kTileF + Nwex - 1;                // window side
    double2* X2 = sm;                                // [2 spins][WX][WX + 1]
    double2* X1 = X2 + 2 * WX * (WX + 1);            // [2 spins][kTileF t2][kTileF + 1 t1]
    double2* A = X1 + 2 * kTileF * (kTileF + 1);     // [kTileF t1][Nwex]
    double2* B = A + kTileF * Nwex;                  // [kTileF t2][Nwex]
    const double w1 = CH == G4_PH_MAGNETIC ? -1.0 : 1.0;  // weight of spin -1 in a, b
    // G(K2, K1) of the tile (the transverse channel pairs the opposite spin)
    for (int t = threadIdx.x; t < 2 * kTileF * kTileF; t += blockDim.x) {
        const int sp = t / (kTileF * kTileF), r = t % (kTileF * kTileF);
        const int a2 = r / kTileF, a1 = r % kTileF;
        const int m1 = n1_0 + a1, m2 = n2_0 + a2;
        const int gs = CH == G4_PH_TRANSVERSE ? 1 - sp : sp;
        X1[(sp * kTileF + a2) * (kTileF + 1) + a1] =
            (m1 < Nw2 && m2 < Nw2) ? G[gs * NN + (size_t)(k2 * Nw2 + m2) * N + k1 * Nw2 + m1]
                                   : make_double2(0.0, 0.0);
    }
    for (int q = 0; q < d.Nkex; ++q) {
        const int k1q = kadd[k1 * d.Nc + q], k2q = kadd[k2 * d.Nc + q];
        __syncthreads();  // the previous q's tiles are no longer read
        for (int t = threadIdx.x; t < 2 * WX * WX; t += blockDim.x) {
            const int sp = t / (WX * WX), r = t % (WX * WX);
            const int i = r / WX, j = r % WX;
            const int f1 = n1_0 + i + d.m0, f2 = n2_0 + j + d.m0;  // frequencies n + m
            X2[(sp * WX + i) * (WX + 1) + j] =
                (f1 < Nw2 && f2 < Nw2) ? G[sp * NN + (size_t)(k1q * Nw2 + f1) * N + k2q * Nw2 + f2]
                                       : make_double2(0.0, 0.0);
        }
        if (CH != G4_PH_TRANSVERSE) {
            for (int t = threadIdx.x; t < 2 * kTileF * Nwex; t += blockDim.x) {
                const int side = t / (kTileF * Nwex), r = t % (kTileF * Nwex);
                const int u = r / Nwex, m = r % Nwex;
                const int mg = d.m0 + m;
                double2 v = make_double2(0.0, 0.0);
                if (side == 0) {
                    // a(n1, m) = sum_s w_s G_s((k1 (+) q, n1 + m), (k1, n1))
                    const int nn = n1_0 + u;
                    if (nn < Nw2 && nn + mg < Nw2) {
                        const size_t i0 = (size_t)(k1q * Nw2 + nn + mg) * N + k1 * Nw2 + nn;
                        const double2 g0 = G[i0], g1 = G[NN + i0];
                        v = make_double2(g0.x + w1 * g1.x, g0.y + w1 * g1.y);
                    }
                    A[u * Nwex + m] = v;
                } else {
                    // b(n2, m) = sum_s w_s G_s((k2, n2), (k2 (+) q, n2 + m))
                    const int nn = n2_0 + u;
                    if (nn < Nw2 && nn + mg < Nw2) {
                        const size_t i0 = (size_t)(k2 * Nw2 + nn) * N + k2q * Nw2 + nn + mg;
                        const double2 g0 = G[i0], g1 = G[NN + i0];
                        v = make_double2(g0.x + w1 * g1.x, g0.y + w1 * g1.y);
                    }
                    B[u * Nwex + m] = v;
                }
            }
        }
        __syncthreads();
        if (!live) continue;
        double2* row = acc + ((size_t)(k1 * Nw2 + n1) * N + k2 * Nw2 + n2) * d.NQ + (size_t)q * Nwex;
        for (int m = 0; m < Nwex; ++m) {
            if (n1 + d.m0 + m >= Nw2 || n2 + d.m0 + m >= Nw2) continue;  // structurally zero
            double2 term = make_double2(0.0, 0.0);
            if (CH != G4_PH_TRANSVERSE) term = cmul(A[t1 * Nwex + m], B[t2 * Nwex + m]);
#pragma unroll
            for (int sp = 0; sp < 2; ++sp) {
                const double2 e = cmul(X1[(sp * kTileF + t2) * (kTileF + 1) + t1],
                                       X2[(sp * WX + t1 + m) * (WX + 1) + t2 + m]);
                term.x -= e.x;
                term.y -= e.y;
            }
            double2 o = row[m];
            o.x += sign * term.x;
            o.y += sign * term.y;
            row[m] = o;
        }
    }
}

// out[m][n2][n1][q][k2][k1] = acc[k1][n1][k2][n2][q][m] * inv_s for n2 in
// [n2_0, n2_0 + gridDim.y), written at out + m * out_plane + (n2 - n2_0) * (one
// n2 plane): the whole exported array when out_plane = E / Nwex and n2_0 = 0,
// or a staging block of a few n2 planes per m.  A block owns one (n1, n2, q)
// triple and walks k2 in chunks of KC through shared memory: it reads runs of
// Nwex contiguous entries (all m of one (k1, k2)) and writes runs of KC*Nc
// contiguous entries (one (m, q) plane).
// The value of an accumulator entry: complex128, or a pair of complex64 whose
// sum is the value (compensated FP32 pairs; hi + lo is exact in FP64).
template <bool PAIR>
__device__ __forceinline__ double2 acc_value(const double2* acc, size_t i) {
    if constexpr (PAIR) {
        const float4 a = reinterpret_cast<const float4*>(acc)[i];
        return make_double2((double)a.x + (double)a.z, (double)a.y + (double)a.w);
    } else {
        return acc[i];
    }
}

template <bool PAIR>
__global__ void k_finalize(const double2* __restrict__ acc, double inv_s,
                           double2* __restrict__ out, G4Dims d, int KC, int n2_0,
                           long long out_plane) {
    extern __shared__ double2 tileF[];  // [KC][Nc][Nwex + 1]
    const int n1 = blockIdx.x, n2l = blockIdx.y, q = blockIdx.z;
    const int n2 = n2_0 + n2l;
    const int Nc = d.Nc, Nw2 = d.Nw2, Nwex = d.Nwex, ld = Nwex + 1;
    for (int k20 = 0; k20 < Nc; k20 += KC) {
        const int kc = min(KC, Nc - k20);
        const int cnt = kc * Nc * Nwex;
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int m = t % Nwex;
            const int r = t / Nwex;
            const int k1 = r % Nc, k2l = r / Nc;
            const size_t K1 = (size_t)k1 * Nw2 + n1, K2 = (size_t)(k20 + k2l) * Nw2 + n2;
            tileF[(k2l * Nc + k1) * ld + m] = acc_value<PAIR>(acc, (K1 * d.N + K2) * d.NQ + (size_t)q * Nwex + m);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int r = t % (kc * Nc);       // (k2l, k1), k1 fastest
            const int m = t / (kc * Nc);
            const double2 v = tileF[r * ld + m];
            const size_t o = (size_t)m * out_plane +
                             (((size_t)n2l * Nw2 + n1) * d.Nkex + q) * Nc * Nc + (size_t)k20 * Nc + r;
            out[o] = make_double2(v.x * inv_s, v.y * inv_s);
        }
        __syncthreads();
    }
}

// Fallback for shapes whose (k1, m) plane does not fit in shared memory: one
// thread per output entry of the n2 range, gathering from the accumulator.
template <bool PAIR>
__global__ void k_finalize_gather(const double2* __restrict__ acc, double inv_s,
                                  double2* __restrict__ out, G4Dims d, int n2_0, int n2_cnt,
                                  long long out_plane) {
    const long long cnt = (long long)d.Nwex * n2_cnt * d.Nw2 * d.Nkex * d.Nc * d.Nc;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < cnt;
         o += (long long)gridDim.x * blockDim.x) {
        long long t = o;
        const int k1 = (int)(t % d.Nc); t /= d.Nc;
        const int k2 = (int)(t % d.Nc); t /= d.Nc;
        const int q = (int)(t % d.Nkex); t /= d.Nkex;
        const int n1 = (int)(t % d.Nw2); t /= d.Nw2;
        const int n2l = (int)(t % n2_cnt);
        const int m = (int)(t / n2_cnt);
        const int n2 = n2_0 + n2l;
        const size_t K1 = (size_t)k1 * d.Nw2 + n1, K2 = (size_t)k2 * d.Nw2 + n2;
        const double2 v = acc_value<PAIR>(acc, (K1 * d.N + K2) * d.NQ + (size_t)q * d.Nwex + m);
        const size_t po = (((size_t)n2l * d.Nw2 + n1) * d.Nkex + q) * d.Nc * d.Nc + (size_t)k2 * d.Nc + k1;
        out[(size_t)m * out_plane + po] = make_double2(v.x * inv_s, v.y * inv_s);
    }
}

// Mixed path G build.  One block owns the (row momentum kr, column momentum kc)
// frequency block of one spin: it forms G in FP32, scales it by sqrt(s_r)
// (i sqrt(|s_r|) for a negative sign, so that the product of two entries of
// the same measurement carries s_r), rounds to complex64 into a padded shared
// tile, then writes every frequency-difference diagonal of the block into its
// Nw2-long row (the positions where the row index leaves the grid stay zero):
//   Gd[j][dk][dn + Nw2-1][kc][n] = sqrt(s_r) G((kr, n+dn), (kc, n)),  kr = kc (+) dk.
// WRITE = false is the same pass without the tile and the writes: only the
// largest component joins *gmax (the deferred staging's per-measurement pass).
template <bool M64, bool WRITE>
__global__ void __launch_bounds__(256) k_build_G_diag(const void* __restrict__ M,
                                                      const double2* __restrict__ G0, double sign,
                                                      float2* __restrict__ Gd,
                                                      const int* __restrict__ ksub, G4Dims d,
                                                      unsigned* __restrict__ gmax) {
    extern __shared__ float2 tile[];  // [Nw2][Nw2+2] (WRITE), then G0 of the block's rows [Nw2]
    const int kc = blockIdx.x, kr = blockIdx.y, sp = blockIdx.z;
    const int Nw2 = d.Nw2, N = d.N, ld = Nw2 + 2;
    const size_t NN = (size_t)N * N;
    float2* g0row = tile + (WRITE ? Nw2 * ld : 0);
    // complex64 storage: form G in FP32 (three roundings, below the storage rounding scale)
    const g4gt::SignFactor sf = g4gt::sign_factor(sign);
    for (int i = threadIdx.x; i < Nw2; i += blockDim.x) {
        const double2 g = G0[sp * N + kr * Nw2 + i];
        g0row[i] = make_float2((float)g.x, (float)g.y);
    }
    __syncthreads();
    // Thread layout: a fixed column j = tid % Nw2 and rows i = tid / Nw2 + RPB*k
    // (RPB rows per sweep), so no per-element division; U independent loads of
    // M per thread are in flight before any is used (eight 8-byte loads of a
    // complex64 M or four 16-byte loads of a complex128 one; sixteen with a
    // register cap for three blocks per SM measured 12% slower).
    const int RPB = blockDim.x / Nw2 > 0 ? blockDim.x / Nw2 : 1;
    const int j = threadIdx.x % Nw2, i0 = threadIdx.x / Nw2;
    const bool lane_ok = i0 < RPB;  // threads beyond RPB*Nw2 (Nw2 not dividing the block) idle
    const double2 gj64 = G0[sp * N + kc * Nw2 + j];
    const float2 gj = make_float2((float)gj64.x, (float)gj64.y);
    const size_t mbase = sp * NN + (size_t)(kr * Nw2) * N + kc * Nw2 + j;
    constexpr int U = M64 ? 8 : 4;
    float vmax = 0.f;
    // M entries as loaded: complex64 stays complex64, complex128 is narrowed below
    using MV = typename std::conditional<M64, float2, double2>::type;
    if (lane_ok) {
        for (int ib = i0; ib < Nw2; ib += U * RPB) {
            MV mv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = ib + u * RPB;
                if (i < Nw2) mv[u] = reinterpret_cast<const MV*>(M)[mbase + (size_t)i * N];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = ib + u * RPB;
                if (i >= Nw2) break;
                const float2 v = g4gt::g_tilde(g0row[i], g4gt::to_c64(mv[u]), gj, kr == kc && i == j, sf);
                if constexpr (WRITE) tile[i * ld + j] = v;
                vmax = fmaxf(vmax, fmaxf(fabsf(v.x), fabsf(v.y)));
            }
        }
    }
    // the block's largest component joins the batch's maximum (non-negative
    // FP32 values order like their bit patterns)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(gmax, __float_as_uint(vmax));
    if constexpr (!WRITE) return;
    __syncthreads();
    // Only the in-grid part of each diagonal is written; the out-of-grid part
    // of every row is zero once and for all (cleared when the handle is made).
    const int dk = ksub[kr * d.Nc + kc];
    float2* base = Gd + (((size_t)sp * d.Nc + dk) * d.ndn) * ((size_t)d.Nc * Nw2);
    if (lane_ok) {
        const int n = j;
        for (int dnI = i0; dnI < d.ndn; dnI += RPB) {
            const int row = n + dnI - (Nw2 - 1);
            if (row >= 0 && row < Nw2)
                base[((size_t)dnI * d.Nc + kc) * Nw2 + n] = tile[row * ld + n];
        }
    }
}

int grid_for(size_t work, int block) {
    size_t g = (work + block - 1) / block;
    if (g > (size_t)152 * 64) g = (size_t)152 * 64;
    return (int)(g ? g : 1);
}

}  // namespace

cudaError_t launch_build_G_fp64(const void* M, bool m64, const double2* G0, double2* G, int N,
                                cudaStream_t s) {
    const size_t total = 2 * (size_t)N * N;
    const int g = grid_for(total, 256);
    if (m64)
        k_build_G_fp64<true><<<g, 256, 0, s>>>(M, G0, G, N);
    else
        k_build_G_fp64<false><<<g, 256, 0, s>>>(M, G0, G, N);
    return cudaGetLastError();
}

cudaError_t launch_update_fp64(const double2* G, double sign, double2* acc, const int* kadd,
                               const int* ksub, const G4Dims& d, cudaStream_t s) {
    if (d.ch != G4_PP_UPDOWN && d.Nwex <= kTileWex && (long long)d.Nc * d.Nc <= 65535) {
        const int nt = (d.Nw2 + kTileF - 1) / kTileF;
        const int WX = kTileF + d.Nwex - 1;
        const size_t smem = (2 * (size_t)WX * (WX + 1) + 2 * kTileF * (kTileF + 1) +
                             2 * (size_t)kTileF * d.Nwex) * sizeof(double2);
        const dim3 grid(nt * nt, d.Nc * d.Nc);
        cudaError_t e;
        switch (d.ch) {
            case G4_PH_DENSITY:
                if ((e = raise_smem_limit(k_update_fp64_tiled<G4_PH_DENSITY>)) != cudaSuccess) return e;
                k_update_fp64_tiled<G4_PH_DENSITY><<<grid, kTileF * kTileF, smem, s>>>(G, sign, acc, kadd, d);
                break;
            case G4_PH_TRANSVERSE:
                if ((e = raise_smem_limit(k_update_fp64_tiled<G4_PH_TRANSVERSE>)) != cudaSuccess) return e;
                k_update_fp64_tiled<G4_PH_TRANSVERSE><<<grid, kTileF * kTileF, smem, s>>>(G, sign, acc, kadd, d);
                break;
            default:
                if ((e = raise_smem_limit(k_update_fp64_tiled<G4_PH_MAGNETIC>)) != cudaSuccess) return e;
                k_update_fp64_tiled<G4_PH_MAGNETIC><<<grid, kTileF * kTileF, smem, s>>>(G, sign, acc, kadd, d);
        }
        return cudaGetLastError();
    }
    const int per = d.N * d.NQ;
    int gx = (per + 255) / 256;
    if (gx > 64) gx = 64;
    dim3 grid(gx, d.N);
    switch (d.ch) {
        case G4_PP_UPDOWN:
            k_update_fp64<G4_PP_UPDOWN><<<grid, 256, 0, s>>>(G, sign, acc, kadd, ksub, d);
            break;
        case G4_PH_DENSITY:
            k_update_fp64<G4_PH_DENSITY><<<grid, 256, 0, s>>>(G, sign, acc, kadd, ksub, d);
            break;
        case G4_PH_TRANSVERSE:
            k_update_fp64<G4_PH_TRANSVERSE><<<grid, 256, 0, s>>>(G, sign, acc, kadd, ksub, d);
            break;
        default:
            k_update_fp64<G4_PH_MAGNETIC><<<grid, 256, 0, s>>>(G, sign, acc, kadd, ksub, d);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double2* acc, bool pair, double inv_s, double2* out,
                            const G4Dims& d, int n2_0, int n2_cnt, long long out_plane,
                            cudaStream_t s) {
    int KC = (int)((24 * 1024) / ((size_t)d.Nc * (d.Nwex + 1) * sizeof(double2)));
    KC = KC < 1 ? 1 : (KC > d.Nc ? d.Nc : KC);
    const size_t smem = (size_t)KC * d.Nc * (d.Nwex + 1) * sizeof(double2);
    cudaError_t e;
    if (smem > 96 * 1024) {
        const long long cnt = (long long)d.Nwex * n2_cnt * d.Nw2 * d.Nkex * d.Nc * d.Nc;
        long long blocks = (cnt + 255) / 256;
        if (blocks > 152 * 64) blocks = 152 * 64;
        auto* k = pair ? k_finalize_gather<true> : k_finalize_gather<false>;
        k<<<(int)blocks, 256, 0, s>>>(acc, inv_s, out, d, n2_0, n2_cnt, out_plane);
    } else {
        auto* k = pair ? k_finalize<true> : k_finalize<false>;
        if (smem > 48 * 1024) {
            e = raise_smem_limit(k);
            if (e != cudaSuccess) return e;
        }
        k<<<dim3(d.Nw2, n2_cnt, d.Nkex), 256, smem, s>>>(acc, inv_s, out, d, KC, n2_0, out_plane);
    }
    return cudaGetLastError();
}

cudaError_t launch_build_G_diag(const void* M, bool m64, const double2* G0, double sign,
                                float2* Gd_slot, const int* ksub, const G4Dims& d,
                                unsigned* gmax, cudaStream_t s) {
    // Gd_slot == nullptr: the largest-|G~| pass alone
    const bool write = Gd_slot != nullptr;
    const size_t smem = ((write ? (size_t)d.Nw2 * (d.Nw2 + 2) : 0) + d.Nw2) * sizeof(float2);
    dim3 grid(d.Nc, d.Nc, 2);
    auto* k = m64 ? (write ? k_build_G_diag<true, true> : k_build_G_diag<true, false>)
                  : (write ? k_build_G_diag<false, true> : k_build_G_diag<false, false>);
    cudaError_t e = raise_smem_limit(k);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, s>>>(M, G0, sign, Gd_slot, ksub, d, gmax);
    return cudaGetLastError();
}
