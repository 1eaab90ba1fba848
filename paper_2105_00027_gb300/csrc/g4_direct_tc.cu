// Direct term of the particle-hole magnetic G4 update:
//   Dir(K1, K2, Q) = sum_r a_r(K1) b_r(K2),
//   a_r(K1) = s_r sum_s s G_s(K1+Q, K1),  b_r(K2) = sum_s s G_s(K2, K2+Q).
// For fixed Q this is a sum of rank-1 outer products over the batch, i.e. a
// GEMM with the batch as its K dimension.  Operands come from k_pack_direct
// (TF32 hi/lo split, real embedding of the complex product).
#include "g4_internal.h"

namespace {

__global__ void k_direct_simt(const float* __restrict__ Ah, const float* __restrict__ Al,
                              const float* __restrict__ Bh, const float* __restrict__ Bl, int Bp,
                              double2* __restrict__ acc, G4Dims d) {
    const long long per = (long long)d.N * d.NQ;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < d.E;
         e += (long long)gridDim.x * blockDim.x) {
        const long long K1 = e / per, rem = e - K1 * per;
        const int K2 = (int)(rem / d.NQ), Qi = (int)(rem - (long long)K2 * d.NQ);
        const size_t ra = ((size_t)Qi * d.N + K1) * (2 * Bp);
        const size_t rb0 = (((size_t)Qi * 2 + 0) * d.N + K2) * (2 * Bp);
        const size_t rb1 = (((size_t)Qi * 2 + 1) * d.N + K2) * (2 * Bp);
        float re = 0.f, im = 0.f;
        for (int kk = 0; kk < 2 * Bp; ++kk) {
            const float ah = Ah[ra + kk], al = Al[ra + kk];
            re += ah * Bh[rb0 + kk] + ah * Bl[rb0 + kk] + al * Bh[rb0 + kk];
            im += ah * Bh[rb1 + kk] + ah * Bl[rb1 + kk] + al * Bh[rb1 + kk];
        }
        double2 o = acc[e];
        o.x += re;
        o.y += im;
        acc[e] = o;
    }
}

}  // namespace

g4_status direct_prepare(g4_ctx*) { return G4_OK; }

g4_status direct_run(g4_ctx* h, int) {
    long long blocks = (h->d.E + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_direct_simt<<<(int)blocks, 256, 0, h->stream>>>(h->Ah, h->Al, h->Bh, h->Bl, h->Bp, h->acc,
                                                      h->d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return g4_cuda_fail(h, e, "direct launch");
    return G4_OK;
}

void direct_release(g4_ctx*) {}
