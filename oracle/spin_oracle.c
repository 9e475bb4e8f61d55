/*
 * spin_oracle.c -- plain FP64 CPU oracle for the random-phase pure-state method
 * of Alvarez, Danieli, Levstein & Pastawski, "Quantum parallelism as a tool for
 * ensemble spin dynamics calculations" (arXiv:0710.3747).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark compile, load or call this file.  The
 * product library never links or calls it, and the two share no code.
 *
 * What it computes, in the paper's terms:
 *   - the entangled random-phase state of the "Testing the quantum parallelism"
 *     section: spin 1 up, every basis state |Psi_i> of spins 2..M with weight
 *     2^{-(M-1)/2} and an independent phase;
 *   - its evolution under the secular spin-spin Hamiltonian of the "Spin systems
 *     with different coupling networks" section,
 *         H = sum_{i<j} [ a_ij S^z_i S^z_j + b_ij (S^x_i S^x_j + S^y_i S^y_j) ]
 *     (equal to the paper's 1/2 b_ij (I+ I- + I- I+) form), by a symmetric
 *     second-order Trotter-Suzuki product (the paper names the decomposition in
 *     its introduction and summary but fixes neither order nor splitting);
 *   - the local polarization P_11(t) = 2 [W_11(t) - 1/2] (Eq. 2 with m = m' = 1)
 *     read out after every step, normalised by the norm.
 *
 * Conventions: spin n (1-based) is bit n-1 of the basis index x; a set bit is
 * spin up (S^z = +1/2); S = sigma/2; hbar = 1.  A state is 2^M complex
 * amplitudes stored as interleaved (re, im) doubles.
 *
 * Trotter step (splitting "diagonal outside, flip-flops inside"), tau = dt/2:
 *     U(dt) = e^{-i tau D} F_1(tau) ... F_B(tau) F_B(tau) ... F_1(tau) e^{-i tau D}
 * written in the order the factors are applied (D = sum a_ij S^z_i S^z_j,
 * F_k(tau) = exp(-i tau b_k (S^x S^x + S^y S^y)) on bond k, bonds in the order
 * given).  The product is a palindrome, so U(dt)^{-1} = U(-dt).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror & Shaw,  */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4-word counter and */
/* a 2-word key; each round multiplies counter words 0 and 2 by two fixed      */
/* 32-bit multipliers, keeps both halves of the 64-bit products, mixes them    */
/* with the other counter words and the key, and then bumps the key by the     */
/* two Weyl constants.                                                         */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform u in [0,1) for basis index r of spins 2..M: counter (lo r, hi r, 0, 0),
 * key (lo seed, hi seed); the top 53 bits of (out0:out1) scaled by 2^-53. */
double oracle_phase_uniform(uint64_t seed, uint64_t r)
{
    uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(r >> 32), 0u, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    uint64_t bits = ((uint64_t)out[0] << 32) | (uint64_t)out[1];
    return (double)(bits >> 11) * (1.0 / 9007199254740992.0);
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* ------------------------------------------------------------------------ */
/* Initial state: |Psi_ent> = sum_r 2^{-(M-1)/2} e^{i phi_r} |up>_1 (x) |r>,   */
/* phi_r = 2 pi u(seed, r).  Amplitudes with spin 1 down are zero.             */
/* ------------------------------------------------------------------------ */
int oracle_init_random_phase(int M, uint64_t seed, double *psi, int nthreads)
{
    if (M < 1 || M > 40) return 1;
    set_threads(nthreads);
    const int64_t N = (int64_t)1 << M;
    const double amp = pow(2.0, -0.5 * (double)(M - 1));
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        if ((x & 1) == 0) {
            psi[2 * x] = 0.0;
            psi[2 * x + 1] = 0.0;
        } else {
            double phi = ORACLE_TWO_PI * oracle_phase_uniform(seed, (uint64_t)x >> 1);
            psi[2 * x] = amp * cos(phi);
            psi[2 * x + 1] = amp * sin(phi);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Flip-flop bond gate exp(-i tau b (S^x_i S^x_j + S^y_i S^y_j)).              */
/* The operator maps |1_i 0_j> to (b/2)|0_i 1_j> and back and annihilates      */
/* |00>, |11>; so on each pair (x: bit i set, bit j clear; y = x with both     */
/* bits flipped) it is cos(b tau/2) - i sin(b tau/2) sigma_x, and the identity */
/* elsewhere.                                                                  */
/* ------------------------------------------------------------------------ */
void oracle_flipflop(int M, double *psi, int i, int j, double b, double tau, int nthreads)
{
    set_threads(nthreads);
    const double c = cos(0.5 * b * tau), s = sin(0.5 * b * tau);
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    const int64_t npairs = (int64_t)1 << (M - 2);
    const uint64_t bit_i = (uint64_t)1 << i, bit_j = (uint64_t)1 << j;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < npairs; ++k) {
        /* insert a zero at bit lo, then at bit hi: all indices with both bits clear */
        uint64_t t = (uint64_t)k;
        t = ((t >> lo) << (lo + 1)) | (t & (((uint64_t)1 << lo) - 1));
        t = ((t >> hi) << (hi + 1)) | (t & (((uint64_t)1 << hi) - 1));
        const uint64_t x = t | bit_i, y = t | bit_j;
        const double xr = psi[2 * x], xi = psi[2 * x + 1];
        const double yr = psi[2 * y], yi = psi[2 * y + 1];
        /* x' = c x - i s y ;  y' = -i s x + c y */
        psi[2 * x] = c * xr + s * yi;
        psi[2 * x + 1] = c * xi - s * yr;
        psi[2 * y] = c * yr + s * xi;
        psi[2 * y + 1] = c * yi - s * xr;
    }
}

/* Diagonal energy E(x) = sum_{i<j} a_ij s_i s_j, s = +1/2 (bit set) or -1/2. */
double oracle_diag_energy(int M, const double *a, uint64_t x)
{
    double e = 0.0;
    for (int i = 0; i < M; ++i) {
        const double si = ((x >> i) & 1) ? 0.5 : -0.5;
        for (int j = i + 1; j < M; ++j) {
            const double sj = ((x >> j) & 1) ? 0.5 : -0.5;
            e += a[i * M + j] * si * sj;
        }
    }
    return e;
}

/* Phase table ph[x] = exp(-i tau E(x)) (interleaved re, im). */
void oracle_diag_table(int M, const double *a, double tau, double *ph, int nthreads)
{
    set_threads(nthreads);
    const int64_t N = (int64_t)1 << M;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        const double th = -tau * oracle_diag_energy(M, a, (uint64_t)x);
        ph[2 * x] = cos(th);
        ph[2 * x + 1] = sin(th);
    }
}

/* psi[x] <- ph[x] psi[x] */
void oracle_apply_table(int M, double *psi, const double *ph, int nthreads)
{
    set_threads(nthreads);
    const int64_t N = (int64_t)1 << M;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        const double pr = ph[2 * x], pi = ph[2 * x + 1];
        const double vr = psi[2 * x], vi = psi[2 * x + 1];
        psi[2 * x] = pr * vr - pi * vi;
        psi[2 * x + 1] = pr * vi + pi * vr;
    }
}

/* e^{-i tau D} without a table (one energy evaluation per amplitude). */
void oracle_diag(int M, double *psi, const double *a, double tau, int nthreads)
{
    set_threads(nthreads);
    const int64_t N = (int64_t)1 << M;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        const double th = -tau * oracle_diag_energy(M, a, (uint64_t)x);
        const double pr = cos(th), pi = sin(th);
        const double vr = psi[2 * x], vi = psi[2 * x + 1];
        psi[2 * x] = pr * vr - pi * vi;
        psi[2 * x + 1] = pr * vi + pi * vr;
    }
}

/* Populations of spin `site` (1-based): n_up = sum |psi_x|^2 over x with the
 * site's bit set, n_dn over the rest. */
void oracle_site_populations(int M, const double *psi, int site, double *n_up, double *n_dn,
                             int nthreads)
{
    set_threads(nthreads);
    const int64_t N = (int64_t)1 << M;
    const int q = site - 1;
    double up = 0.0, dn = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : up, dn)
    for (int64_t x = 0; x < N; ++x) {
        const double p = psi[2 * x] * psi[2 * x] + psi[2 * x + 1] * psi[2 * x + 1];
        if ((x >> q) & 1) up += p;
        else dn += p;
    }
    *n_up = up;
    *n_dn = dn;
}

/* ------------------------------------------------------------------------ */
/* Evolution: `steps` second-order Trotter steps of size dt.  bonds holds      */
/* nbonds pairs (i, j) of 0-based spin indices in the order of the forward     */
/* half step; b is the M x M flip-flop coupling matrix (row-major), a the      */
/* S^z S^z one.  After step n (1..steps) P[n-1] = (N_up - N_dn)/(N_up + N_dn)  */
/* of spin `site` and norm[n-1] = N_up + N_dn.                                 */
/* The diagonal factor is skipped when every a_ij (i<j) is zero (it is then    */
/* the identity); otherwise its phase table for tau is built once and reused, */
/* which only memoises values the definition recomputes identically.          */
/* ------------------------------------------------------------------------ */
static int has_sz_coupling(int M, const double *a)
{
    for (int i = 0; i < M; ++i)
        for (int j = i + 1; j < M; ++j)
            if (a[i * M + j] != 0.0) return 1;
    return 0;
}

/* One symmetric second-order step: D(tau), forward flip-flops, reversed
 * flip-flops, D(tau); ph is the D(tau) phase table or NULL when D = 0. */
static void trotter_step(int M, double *psi, const double *ph, const double *b, const int32_t *bonds,
                         int nbonds, double tau, int nthreads)
{
    if (ph) oracle_apply_table(M, psi, ph, nthreads);
    for (int k = 0; k < nbonds; ++k) {
        const int i = bonds[2 * k], j = bonds[2 * k + 1];
        oracle_flipflop(M, psi, i, j, b[i * M + j], tau, nthreads);
    }
    for (int k = nbonds - 1; k >= 0; --k) {
        const int i = bonds[2 * k], j = bonds[2 * k + 1];
        oracle_flipflop(M, psi, i, j, b[i * M + j], tau, nthreads);
    }
    if (ph) oracle_apply_table(M, psi, ph, nthreads);
}

int oracle_evolve(int M, double *psi, const double *a, const double *b, const int32_t *bonds,
                  int nbonds, double dt, int64_t steps, int site, double *P, double *norm,
                  int nthreads)
{
    if (M < 2 || site < 1 || site > M || nbonds < 0) return 1;
    const double tau = 0.5 * dt;
    double *ph = NULL;
    if (has_sz_coupling(M, a)) {
        ph = (double *)malloc(sizeof(double) * 2 * ((size_t)1 << M));
        if (!ph) return 2;
        oracle_diag_table(M, a, tau, ph, nthreads);
    }
    for (int64_t n = 0; n < steps; ++n) {
        trotter_step(M, psi, ph, b, bonds, nbonds, tau, nthreads);
        double up, dn;
        oracle_site_populations(M, psi, site, &up, &dn, nthreads);
        if (P) P[n] = (up - dn) / (up + dn);
        if (norm) norm[n] = up + dn;
    }
    free(ph);
    return 0;
}

/* Same evolution, reading out every site: after step n, Pall[n*M + q-1] =
 * (N_up - N_dn)/(N_up + N_dn) of spin q (q = 1..M), the local polarizations
 * P_{q1}(t) of the paper's Eq. 2 with m = 1, and norm[n] = N_up + N_dn. */
int oracle_evolve_all_sites(int M, double *psi, const double *a, const double *b,
                            const int32_t *bonds, int nbonds, double dt, int64_t steps, double *Pall,
                            double *norm, int nthreads)
{
    if (M < 2 || nbonds < 0) return 1;
    const double tau = 0.5 * dt;
    double *ph = NULL;
    if (has_sz_coupling(M, a)) {
        ph = (double *)malloc(sizeof(double) * 2 * ((size_t)1 << M));
        if (!ph) return 2;
        oracle_diag_table(M, a, tau, ph, nthreads);
    }
    for (int64_t n = 0; n < steps; ++n) {
        trotter_step(M, psi, ph, b, bonds, nbonds, tau, nthreads);
        for (int q = 1; q <= M; ++q) {
            double up, dn;
            oracle_site_populations(M, psi, q, &up, &dn, nthreads);
            Pall[n * M + (q - 1)] = (up - dn) / (up + dn);
            if (q == 1 && norm) norm[n] = up + dn;
        }
    }
    free(ph);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Product (unentangled) random state of the "Testing the quantum            */
/* parallelism" section: spin 1 up, every other spin l in                     */
/* (|down> + e^{-i phi_l} |up>)/sqrt(2) with its own random phase:            */
/*   psi_x = 2^{-(M-1)/2} exp(-i sum_{l up in x, l >= 2} phi_l)  (spin 1 up)  */
/* phi_l = 2 pi u_l, u_l = top 53 bits of the first two Philox4x32-10 output  */
/* words for counter (l - 1, 0, 0, 1) (l = 2..M, i.e. bit index l - 1) and   */
/* key (lo seed, hi seed), times 2^-53.                                       */
/* ------------------------------------------------------------------------ */
double oracle_product_uniform(uint64_t seed, int bit)
{
    uint32_t ctr[4] = {(uint32_t)bit, 0u, 0u, 1u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    uint64_t bits = ((uint64_t)out[0] << 32) | (uint64_t)out[1];
    return (double)(bits >> 11) * (1.0 / 9007199254740992.0);
}

int oracle_init_product_phase(int M, uint64_t seed, double *psi, int nthreads)
{
    if (M < 1 || M > 40) return 1;
    set_threads(nthreads);
    double phi[64];
    for (int q = 1; q < M; ++q) phi[q] = ORACLE_TWO_PI * oracle_product_uniform(seed, q);
    const int64_t N = (int64_t)1 << M;
    const double amp = pow(2.0, -0.5 * (double)(M - 1));
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        if ((x & 1) == 0) {
            psi[2 * x] = 0.0;
            psi[2 * x + 1] = 0.0;
        } else {
            double th = 0.0;
            for (int q = 1; q < M; ++q)
                if ((x >> q) & 1) th -= phi[q];
            psi[2 * x] = amp * cos(th);
            psi[2 * x + 1] = amp * sin(th);
        }
    }
    return 0;
}
