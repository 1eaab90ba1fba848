/*
 * g4_oracle.c -- plain, slow CPU oracle for the G4 measurement step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * load or call this file: only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA library.
 *
 * Everything is complex128 (C99 `double complex`), written as the definitions
 * read, with no blocking, fusion or reordering:
 *
 *   G_sigma(K1,K2) = G0_sigma(K1) d(K1,K2) - G0_sigma(K1) M_sigma(K1,K2) G0_sigma(K2)
 *       the measured single-particle Green's function of one configuration
 *       (Sec. 2: each walker produces G_sigma for the accumulator; the
 *       diagonal-scaling form is the reading used by this library because G0
 *       is diagonal in K).
 *
 *   G4(K1,K2,Q) += s_r [ (sum_s s G_s(K1+Q,K1)) (sum_s' s' G_s'(K2,K2+Q))
 *                        - sum_s G_s(K2,K1) G_s(K1+Q,K2+Q) ]
 *       the particle-hole magnetic counterpart of the accumulation of Eq. (1)
 *       (Sec. 2.1): Wick's theorem applied to
 *       sum_{s,s'} s s' < c_{K1+Q,s} c+_{K1,s} c_{K2,s'} c+_{K2+Q,s'} >
 *       for a spin-diagonal G.  A G entry whose row or column leaves the
 *       frequency grid is zero.
 *
 *   G4 /= sum_r s_r      (sign-weighted Monte Carlo average).
 *
 * The step before: g4o_nfft gives M from a vertex configuration by the
 * non-uniform Fourier transform (see the comment at the function).
 *
 * Other channels (g4o_accumulate_ch), each Wick's theorem for its correlator:
 *   particle-particle up-down, the accumulation printed as Eq. (1) (Sec. 2.1):
 *     sum_s G_s(Q-K2, Q-K1) G_-s(K2, K1)        (Q-K: momentum q (-) k,
 *                                                 frequency nu_m - w_n)
 *   particle-hole density:  as the magnetic form without the spin weights s, s'
 *   particle-hole transverse: - sum_s G_-s(K2,K1) G_s(K1+Q,K2+Q)
 *
 * Index conventions (shared with the library only through the header text, not
 * code): K = k*Nw2 + n with momentum k = kx + Lx*ky in [0,Nc) and frequency
 * index n in [0,Nw2), Nw2 = 2*Nw, w_n = (2(n-Nw)+1) pi / beta.
 * K+Q = (k (+) q, n+m) where (+) adds lattice momenta componentwise mod Lx, Ly.
 * Complex arrays are interleaved (re, im) doubles.
 *
 * Output slabs: for a list of selected transfers Q_s = (q_s, m_s), the oracle
 * writes slab[s][n2][n1][k2][k1] -- the exported G4 layout restricted to one
 * (q, m) pair.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int Lx, Ly;  /* cluster shape, Nc = Lx * Ly */
    int Nw;      /* number of positive fermionic frequencies (grid is 2*Nw) */
    int Nwex;    /* number of bosonic transfer frequencies, m = 0..Nwex-1 */
    int Nkex;    /* number of transfer momenta, q = 0..Nkex-1 */
} g4o_dims;

/* Lattice momentum addition: componentwise modulo the cluster shape. */
static int kplus(const g4o_dims* d, int a, int b) {
    int ax = a % d->Lx, ay = a / d->Lx;
    int bx = b % d->Lx, by = b / d->Lx;
    return (ax + bx) % d->Lx + d->Lx * ((ay + by) % d->Ly);
}

/* Lattice momentum difference a (-) b. */
static int kminus(const g4o_dims* d, int a, int b) {
    int ax = a % d->Lx, ay = a / d->Lx;
    int bx = b % d->Lx, by = b / d->Lx;
    return (ax - bx + d->Lx) % d->Lx + d->Lx * ((ay - by + d->Ly) % d->Ly);
}

int g4o_kplus(const g4o_dims* d, int a, int b) { return kplus(d, a, b); }

/* G_sigma = G0 d - G0 M G0 for one spin; M, G are N x N row-major. */
void g4o_build_G(int N, const double* M, const double* G0, double* G) {
    const cplx* m = (const cplx*)M;
    const cplx* g0 = (const cplx*)G0;
    cplx* g = (cplx*)G;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            cplx v = -g0[i] * m[(size_t)i * N + j] * g0[j];
            if (i == j) v += g0[i];
            g[(size_t)i * N + j] = v;
        }
}

/*
 * Non-uniform Fourier transform of one spin's vertex configuration (the step
 * that produces M before the G build; Sec. 2: each walker's G_sigma comes from
 * a nonuniform Fourier transform of its configuration):
 *   M(K1, K2) = 1/(beta Nc) sum_{i,j} e^{ i(w_n1 tau_i - k1.x_i)} Mtau_ij
 *                                    e^{-i(w_n2 tau_j - k2.x_j)}
 * with K = k*Nw2 + n, w_n = (2(n-Nw)+1) pi/beta, k.x = 2 pi (kx ix/Lx + ky iy/Ly)
 * for momentum k = kx + Lx ky and site x = ix + Lx iy.  n vertices at times
 * tau[i] and sites site[i]; Mtau is n x n row-major; M is N x N row-major.
 * Evaluated entry by entry as the double sum (K1 x K2 x i x j).
 */
void g4o_nfft(const g4o_dims* d, double beta, int n, const double* tau, const int* site,
              const double* Mtau, double* M) {
    const int Nc = d->Lx * d->Ly, Nw2 = 2 * d->Nw, N = Nc * Nw2;
    const cplx* mt = (const cplx*)Mtau;
    cplx* out = (cplx*)M;
    const double pi = 3.14159265358979323846;
    for (int K1 = 0; K1 < N; ++K1)
        for (int K2 = 0; K2 < N; ++K2) {
            const int k1 = K1 / Nw2, n1 = K1 % Nw2, k2 = K2 / Nw2, n2 = K2 % Nw2;
            const double w1 = (2.0 * (n1 - d->Nw) + 1.0) * pi / beta;
            const double w2 = (2.0 * (n2 - d->Nw) + 1.0) * pi / beta;
            cplx acc = 0.0;
            for (int i = 0; i < n; ++i) {
                const int xi = site[i] % d->Lx, yi = site[i] / d->Lx;
                const double kx1 = 2.0 * pi * (k1 % d->Lx) / d->Lx, ky1 = 2.0 * pi * (k1 / d->Lx) / d->Ly;
                const double ph1 = w1 * tau[i] - (kx1 * xi + ky1 * yi);
                const cplx e1 = cos(ph1) + I * sin(ph1);
                for (int j = 0; j < n; ++j) {
                    const int xj = site[j] % d->Lx, yj = site[j] / d->Lx;
                    const double kx2 = 2.0 * pi * (k2 % d->Lx) / d->Lx, ky2 = 2.0 * pi * (k2 / d->Lx) / d->Ly;
                    const double ph2 = w2 * tau[j] - (kx2 * xj + ky2 * yj);
                    const cplx e2 = cos(ph2) - I * sin(ph2);
                    acc += e1 * mt[(size_t)i * n + j] * e2;
                }
            }
            out[(size_t)K1 * N + K2] = acc / (beta * Nc);
        }
}

/* One entry M(K1, K2) of the transform above (for sampled checks of large N). */
void g4o_nfft_entries(const g4o_dims* d, double beta, int n, const double* tau, const int* site,
                      const double* Mtau, int count, const int* K1s, const int* K2s, double* vals) {
    const int Nc = d->Lx * d->Ly, Nw2 = 2 * d->Nw;
    const cplx* mt = (const cplx*)Mtau;
    cplx* out = (cplx*)vals;
    const double pi = 3.14159265358979323846;
    for (int e = 0; e < count; ++e) {
        const int K1 = K1s[e], K2 = K2s[e];
        const int k1 = K1 / Nw2, n1 = K1 % Nw2, k2 = K2 / Nw2, n2 = K2 % Nw2;
        const double w1 = (2.0 * (n1 - d->Nw) + 1.0) * pi / beta;
        const double w2 = (2.0 * (n2 - d->Nw) + 1.0) * pi / beta;
        cplx acc = 0.0;
        for (int i = 0; i < n; ++i) {
            const int xi = site[i] % d->Lx, yi = site[i] / d->Lx;
            const double kx1 = 2.0 * pi * (k1 % d->Lx) / d->Lx, ky1 = 2.0 * pi * (k1 / d->Lx) / d->Ly;
            const double ph1 = w1 * tau[i] - (kx1 * xi + ky1 * yi);
            const cplx e1 = cos(ph1) + I * sin(ph1);
            for (int j = 0; j < n; ++j) {
                const int xj = site[j] % d->Lx, yj = site[j] / d->Lx;
                const double kx2 = 2.0 * pi * (k2 % d->Lx) / d->Lx, ky2 = 2.0 * pi * (k2 / d->Lx) / d->Ly;
                const double ph2 = w2 * tau[j] - (kx2 * xj + ky2 * yj);
                const cplx e2 = cos(ph2) - I * sin(ph2);
                acc += e1 * mt[(size_t)i * n + j] * e2;
            }
        }
        out[e] = acc / (beta * Nc);
    }
}

/* G(A,B) with the rule that an index off the frequency grid gives zero. */
static cplx gat(const cplx* G, int Nw2, int N, int ka, int na, int kb, int nb) {
    if (na < 0 || na >= Nw2 || nb < 0 || nb >= Nw2) return 0.0;
    return G[(size_t)(ka * Nw2 + na) * N + (kb * Nw2 + nb)];
}

/*
 * One measurement's signed contribution, added into the selected slabs.
 * Gup, Gdn: N x N each (spin +1, spin -1).  acc: [nsel][Nw2][Nw2][Nc][Nc].
 * channel: 0 particle-hole magnetic, 1 particle-particle up-down (Eq. (1),
 * Sec. 2.1), 2 particle-hole density, 3 particle-hole transverse.
 */
void g4o_accumulate_ch(const g4o_dims* d, const double* Gup, const double* Gdn,
                       double sign, const int* qsel, const int* msel, int nsel,
                       double* acc, int nthreads, int channel) {
    const int Nc = d->Lx * d->Ly, Nw2 = 2 * d->Nw, N = Nc * Nw2;
    const cplx* G[2] = {(const cplx*)Gup, (const cplx*)Gdn};
    const double spin[2] = {+1.0, -1.0};
    cplx* out = (cplx*)acc;
    const size_t slab = (size_t)Nw2 * Nw2 * Nc * Nc;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for collapse(2) schedule(static)
#endif
    for (int s = 0; s < nsel; ++s)
        for (int n1 = 0; n1 < Nw2; ++n1) {
            const int q = qsel[s], m = msel[s];
            for (int k1 = 0; k1 < Nc; ++k1)
                for (int n2 = 0; n2 < Nw2; ++n2)
                    for (int k2 = 0; k2 < Nc; ++k2) {
                        const int k1q = kplus(d, k1, q), k2q = kplus(d, k2, q);
                        cplx term = 0.0;
                        if (channel == 1) {
                            /* Q - K: momentum q (-) k, frequency nu_m - w_n, i.e. index
                               m + Nw2 - 1 - n */
                            const int qk1 = kminus(d, q, k1), qk2 = kminus(d, q, k2);
                            const int f1 = m + Nw2 - 1 - n1, f2 = m + Nw2 - 1 - n2;
                            for (int sp = 0; sp < 2; ++sp)
                                term += gat(G[sp], Nw2, N, qk2, f2, qk1, f1) *
                                        gat(G[1 - sp], Nw2, N, k2, n2, k1, n1);
                        } else if (channel == 3) {
                            for (int sp = 0; sp < 2; ++sp)
                                term -= gat(G[1 - sp], Nw2, N, k2, n2, k1, n1) *
                                        gat(G[sp], Nw2, N, k1q, n1 + m, k2q, n2 + m);
                        } else {
                            cplx a = 0.0, b = 0.0, exc = 0.0;
                            for (int sp = 0; sp < 2; ++sp) {
                                const double w = channel == 0 ? spin[sp] : 1.0;
                                a += w * gat(G[sp], Nw2, N, k1q, n1 + m, k1, n1);
                                b += w * gat(G[sp], Nw2, N, k2, n2, k2q, n2 + m);
                                exc += gat(G[sp], Nw2, N, k2, n2, k1, n1) *
                                       gat(G[sp], Nw2, N, k1q, n1 + m, k2q, n2 + m);
                            }
                            term = a * b - exc;
                        }
                        out[s * slab + (((size_t)n2 * Nw2 + n1) * Nc + k2) * Nc + k1] += sign * term;
                    }
        }
}

/* Particle-hole magnetic channel (the form the library's default handle computes). */
void g4o_accumulate(const g4o_dims* d, const double* Gup, const double* Gdn,
                    double sign, const int* qsel, const int* msel, int nsel,
                    double* acc, int nthreads) {
    g4o_accumulate_ch(d, Gup, Gdn, sign, qsel, msel, nsel, acc, nthreads, 0);
}

/*
 * Whole run on selected slabs: R measurements, M = [R][2][N][N], G0 = [2][N],
 * signs[R].  Writes the normalised slabs and the sign sum.  Returns 0, or 5
 * when the sign sum is zero (the unnormalised sums are then left in `out`).
 */
int g4o_run_ch(const g4o_dims* d, int R, const double* M, const double* G0,
               const double* signs, const int* qsel, const int* msel, int nsel,
               double* out, double* sign_sum, int nthreads, int channel) {
    const int Nc = d->Lx * d->Ly, Nw2 = 2 * d->Nw, N = Nc * Nw2;
    const size_t nn = (size_t)N * N;
    const size_t total = (size_t)nsel * Nw2 * Nw2 * Nc * Nc;
    double* G = (double*)malloc(2 * nn * 2 * sizeof(double));
    if (!G) return 2;
    memset(out, 0, total * 2 * sizeof(double));
    double S = 0.0;
    for (int r = 0; r < R; ++r) {
        for (int sp = 0; sp < 2; ++sp)
            g4o_build_G(N, M + ((size_t)r * 2 + sp) * nn * 2, G0 + (size_t)sp * N * 2,
                        G + (size_t)sp * nn * 2);
        g4o_accumulate_ch(d, G, G + nn * 2, signs[r], qsel, msel, nsel, out, nthreads, channel);
        S += signs[r];
    }
    free(G);
    *sign_sum = S;
    if (S == 0.0) return 5;
    cplx* o = (cplx*)out;
    for (size_t i = 0; i < total; ++i) o[i] /= S;
    return 0;
}

int g4o_run(const g4o_dims* d, int R, const double* M, const double* G0,
            const double* signs, const int* qsel, const int* msel, int nsel,
            double* out, double* sign_sum, int nthreads) {
    return g4o_run_ch(d, R, M, G0, signs, qsel, msel, nsel, out, sign_sum, nthreads, 0);
}
