// Exchange term of the particle-hole magnetic G4 update (the second product
// of the accumulation of Eq. (1), Sec. 2.1, in this channel):
//
//   Exc(K1, K2, Q) = sum_r s_r sum_s G_s(K2, K1) G_s(K1+Q, K2+Q).
//
// For a fixed difference D = K2 - K1 = (dk, dn) this is a banded outer
// product over the batch index j = (r, s):
//
//   Exc(K1, K1+D, Q) = sum_j u_j(K1) w_j(K1+Q),
//   u_j(K1) = s_r G_s(K1+D, K1)      (the D-th diagonal of G, indexed by column)
//   w_j(P)  = G_s(P, P+D)            (the -D-th diagonal, indexed by column P+D)
//
// so a thread that owns one momentum pair (k1, q) and a window of TN
// frequencies n1 times MW transfers m needs TN + (TN+MW-1) complex loads per j
// for TN*MW complex multiply-adds (register tiling).  The block stages u for
// every k1 and w for the block's momenta p = k1 (+) q in shared memory from
// the diagonal-major G (complex64) written by the G build; threads of a warp
// share p, so their w reads are broadcasts.  FP32 accumulation over the whole
// batch, then one FP64 read-modify-write of the accumulator:
//   acc[K1][K2][q][m] -= Exc.
#include <algorithm>

#include "g4_internal.h"

namespace {

constexpr int kThreads = 256;

struct XParams {
    const float2* Gd;      // [2*batch][Nc][ndn][Nc][Nw2]
    const float* slot_s;   // [batch]
    const int* pairs;      // (k1 | q << 16), sorted by p = k1 (+) q
    const int* kadd;
    const int* ksub;
    double2* acc;
    G4Dims d;
    int npairs;
    int nj;                // 2 * staged
    int nwin;              // windows per diagonal
    int nmc;               // m chunks
    int JC;                // j per shared-memory stage
};

template <int TN, int MW>
__global__ void __launch_bounds__(kThreads) k_exchange(XParams P) {
    constexpr int UW = TN + 2;            // padded u row (complex)
    constexpr int WW = TN + MW + 1;       // padded w row (complex), >= TN + MW - 1
    extern __shared__ float2 smem[];
    const G4Dims& d = P.d;
    const int Nw2 = d.Nw2, Nc = d.Nc;

    const int dk = blockIdx.z / P.nmc, mc = blockIdx.z - dk * P.nmc;
    const int m0 = mc * MW;
    const int dnI = blockIdx.y / P.nwin, win = blockIdx.y - dnI * P.nwin;
    const int dn = dnI - (Nw2 - 1);
    const int a = win * TN;
    const int lo = max(a, max(0, -dn)), hi = min(a + TN, min(Nw2, Nw2 - dn));
    if (lo >= hi) return;

    const int pi0 = blockIdx.x * kThreads;
    const int pi = pi0 + threadIdx.x;
    const bool active = pi < P.npairs;
    const int plast = min(P.npairs, pi0 + kThreads) - 1;
    const int pair0 = P.pairs[pi0], pairL = P.pairs[plast];
    const int pfirst = P.kadd[(pair0 & 0xffff) * Nc + (pair0 >> 16)];
    const int plastv = P.kadd[(pairL & 0xffff) * Nc + (pairL >> 16)];
    const int nP = plastv - pfirst + 1;

    int k1 = 0, q = 0, pl = 0;
    if (active) {
        const int pr = P.pairs[pi];
        k1 = pr & 0xffff;
        q = pr >> 16;
        pl = P.kadd[k1 * Nc + q] - pfirst;
    }
    const int dkn = P.ksub[0 * Nc + dk];           // (-)dk
    const int dnIneg = 2 * (Nw2 - 1) - dnI;        // diagonal -dn
    const size_t jstride = (size_t)Nc * d.ndn * Nc * Nw2;
    const size_t ubase = ((size_t)dk * d.ndn + dnI) * Nc * Nw2;
    const size_t wbase = ((size_t)dkn * d.ndn + dnIneg) * Nc * Nw2;

    float2* su = smem;                              // [JC][Nc][UW]
    float2* sw = smem + (size_t)P.JC * Nc * UW;     // [JC][nP][WW]

    float2 acc[TN][MW];
#pragma unroll
    for (int t = 0; t < TN; ++t)
#pragma unroll
        for (int mm = 0; mm < MW; ++mm) acc[t][mm] = make_float2(0.f, 0.f);

    for (int j0 = 0; j0 < P.nj; j0 += P.JC) {
        const int jc = min(P.JC, P.nj - j0);
        __syncthreads();
        // stage u: s_r * Gd[j][dk][dnI][k1][a + t]
        for (int e = threadIdx.x; e < jc * Nc * TN; e += kThreads) {
            const int t = e % TN, r2 = e / TN, kk = r2 % Nc, jj = r2 / Nc;
            const int j = j0 + jj;
            float2 v = make_float2(0.f, 0.f);
            if (a + t < Nw2) {
                v = P.Gd[(size_t)j * jstride + ubase + (size_t)kk * Nw2 + a + t];
                const float s = P.slot_s[j >> 1];
                v.x *= s;
                v.y *= s;
            }
            su[((size_t)jj * Nc + kk) * UW + t] = v;
        }
        // stage w: Gd[j][(-)dk][-dn][p (+) dk][pn + dn], pn = a + m0 + t
        for (int e = threadIdx.x; e < jc * nP * (TN + MW - 1); e += kThreads) {
            const int t = e % (TN + MW - 1), r2 = e / (TN + MW - 1), pp = r2 % nP, jj = r2 / nP;
            const int j = j0 + jj;
            const int pmom = pfirst + pp;
            const int col = a + m0 + t + dn;
            float2 v = make_float2(0.f, 0.f);
            if (col >= 0 && col < Nw2) {
                const int kc = P.kadd[pmom * Nc + dk];
                v = P.Gd[(size_t)j * jstride + wbase + (size_t)kc * Nw2 + col];
            }
            sw[((size_t)jj * nP + pp) * WW + t] = v;
        }
        __syncthreads();
        if (active) {
            for (int jj = 0; jj < jc; ++jj) {
                const float2* ur = su + ((size_t)jj * Nc + k1) * UW;
                const float2* wr = sw + ((size_t)jj * nP + pl) * WW;
                float2 u[TN], w[TN + MW - 1];
#pragma unroll
                for (int t = 0; t < TN; ++t) u[t] = ur[t];
#pragma unroll
                for (int t = 0; t < TN + MW - 1; ++t) w[t] = wr[t];
#pragma unroll
                for (int t = 0; t < TN; ++t)
#pragma unroll
                    for (int mm = 0; mm < MW; ++mm) {
                        const float2 x = u[t], y = w[t + mm];
                        acc[t][mm].x = fmaf(x.x, y.x, acc[t][mm].x);
                        acc[t][mm].y = fmaf(x.x, y.y, acc[t][mm].y);
                        acc[t][mm].x = fmaf(-x.y, y.y, acc[t][mm].x);
                        acc[t][mm].y = fmaf(x.y, y.x, acc[t][mm].y);
                    }
            }
        }
    }
    if (!active) return;
    const int k2 = P.kadd[k1 * Nc + dk];
#pragma unroll
    for (int t = 0; t < TN; ++t) {
        const int n1 = a + t;
        if (n1 < lo || n1 >= hi) continue;
        const size_t K1 = (size_t)k1 * Nw2 + n1, K2 = (size_t)k2 * Nw2 + n1 + dn;
        double2* row = P.acc + (K1 * d.N + K2) * d.NQ + (size_t)q * d.Nwex + m0;
#pragma unroll
        for (int mm = 0; mm < MW; ++mm) {
            if (m0 + mm >= d.Nwex) break;
            double2 o = row[mm];
            o.x -= (double)acc[t][mm].x;
            o.y -= (double)acc[t][mm].y;
            row[mm] = o;
        }
    }
}

struct Cfg {
    int TN, MW;
};

Cfg choose(const G4Dims& d) {
    int MW = 1;
    while (MW < d.Nwex && MW < 8) MW *= 2;
    return Cfg{64 / MW, MW};
}

template <int TN, int MW>
g4_status run_cfg(g4_ctx* h, int staged) {
    const G4Dims& d = h->d;
    XParams P;
    P.Gd = h->Gd;
    P.slot_s = h->slot_s;
    P.pairs = h->pairs;
    P.kadd = h->kadd;
    P.ksub = h->ksub;
    P.acc = h->acc;
    P.d = d;
    P.npairs = h->npairs;
    P.nj = 2 * staged;
    P.nwin = (d.Nw2 + TN - 1) / TN;
    P.nmc = (d.Nwex + MW - 1) / MW;
    const int nPmax = std::min(d.Nc, kThreads);
    const size_t per_j = ((size_t)d.Nc * (TN + 2) + (size_t)nPmax * (TN + MW + 1)) * sizeof(float2);
    int JC = (int)std::max<size_t>(1, (48 * 1024) / per_j);
    JC = std::min(JC, 16);
    P.JC = JC;
    const size_t smem = per_j * JC;
    cudaError_t e = cudaFuncSetAttribute(k_exchange<TN, MW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange smem attribute");
    dim3 grid((h->npairs + kThreads - 1) / kThreads, d.ndn * P.nwin, d.Nc * P.nmc);
    k_exchange<TN, MW><<<grid, kThreads, smem, h->stream>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "exchange launch");
    return G4_OK;
}

}  // namespace

g4_status exchange_prepare(g4_ctx* h) {
    const G4Dims& d = h->d;
    // (k1, q) pairs sorted by p = k1 (+) q, then k1
    std::vector<int> kadd((size_t)d.Nc * d.Nc);
    for (int a = 0; a < d.Nc; ++a)
        for (int b = 0; b < d.Nc; ++b) {
            const int ax = a % d.Lx, ay = a / d.Lx, bx = b % d.Lx, by = b / d.Lx;
            kadd[(size_t)a * d.Nc + b] = (ax + bx) % d.Lx + d.Lx * ((ay + by) % d.Ly);
        }
    std::vector<int> pairs;
    for (int p = 0; p < d.Nc; ++p)
        for (int k1 = 0; k1 < d.Nc; ++k1)
            for (int q = 0; q < d.Nkex; ++q)
                if (kadd[(size_t)k1 * d.Nc + q] == p) pairs.push_back(k1 | (q << 16));
    h->npairs = (int)pairs.size();
    cudaError_t e = cudaMalloc((void**)&h->pairs, pairs.size() * sizeof(int));
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "cudaMalloc pairs");
    h->bytes += pairs.size() * sizeof(int);
    e = cudaMemcpy(h->pairs, pairs.data(), pairs.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "pairs upload");
    return G4_OK;
}

g4_status exchange_run(g4_ctx* h, int staged) {
    const Cfg c = choose(h->d);
    if (c.MW == 8) return run_cfg<8, 8>(h, staged);
    if (c.MW == 4) return run_cfg<16, 4>(h, staged);
    if (c.MW == 2) return run_cfg<32, 2>(h, staged);
    return run_cfg<64, 1>(h, staged);
}

void exchange_release(g4_ctx*) {}
