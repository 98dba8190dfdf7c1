/*
 * lll_oracle.c -- plain, slow FP64 CPU oracle of the Levy LIBOR Monte Carlo.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark are the only callers.  This file shares no
 * code, header, table or constant generator with the CUDA library; both sides
 * only read the same seeded inputs.
 *
 * Paper: A. Papapantoleon, D. Skovmand, "Numerical Methods for the Levy LIBOR
 * model" (arXiv 1006.3340).  What is computed, in the paper's order:
 *   - Section 2, Eq. (log-LIB-SIE) / Section 3, Eq. (log-LIB-SDE-2):
 *     Z(t,T_i) = log L(t,T_i), dZ = b dt + lambda dH, advanced by log-Euler
 *     steps with the drift and lambda taken at the left point of each step.
 *   - Eq. (LIBOR-drift-PT) with the factors of Eq. (Levy-LIBOR-beta): the
 *     drift b(s,T_i), written out directly as the product over l = i+1..n
 *     inside the integral against the Levy measure.  The integral is the
 *     caller's quadrature: int g dF ~= sum_j W_j g(x_j) / x_j^2, where the
 *     W_j integrate against x^2 nu(x) dx.
 *   - Eq. (Picard-2): Z^(1) = Z(0) + int b(s; Z(0)) ds + int lambda dH, and
 *     Eq. (bdrift): the Picard drift evaluated at Z^(1).
 *   - Frozen drift (Section 1, Section 3.2): L^0 = exp(Z^(1)).
 *   - Eq. (caplet): caplet payoffs under the terminal measure.
 *   - Section 4: NIG driver drawn as a normal variance-mean mixture with an
 *     inverse-Gaussian mixing variable (the paper points to the standard
 *     method); the IG variable follows Michael, Schucany & Haas (1976).
 *   - Counter-based uniforms: Philox-4x32-10 of Salmon, Moraes, Dror & Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
 *
 * Tenor convention: N accrual dates, n = N-1 simulated rates L_1..L_n, the
 * spot rate L_0 known at t = 0, terminal date T_N = T_*, so the paper's N is
 * n here.  lam[k*n + (l-1)] = lambda(t_k, T_l).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_FULL 0
#define ORACLE_PICARD 1
#define ORACLE_FROZEN 3

typedef struct {
    int32_t N, s, Q, driver; /* driver: 0 = NIG, 1 = Brownian (c = 1, no jumps) */
    double delta, alpha, beta, dbar, mu; /* mu: NaN selects the martingale value */
    const double *L0;  /* [N]   L(0,T_m), m = 0..N-1 */
    const double *lam; /* [n*s][n] */
    const double *x;   /* [Q] quadrature nodes */
    const double *W;   /* [Q] weights against x^2 nu(x) dx */
} oracle_model;

/* ------------------------------------------------------------------------- */
/* Philox-4x32-10 (Salmon et al. 2011): ten rounds of two 32x32->64 bit      */
/* multiplications of the even words, XOR of the high halves into the odd    */
/* words and the round key, then a word permutation; the key is bumped by    */
/* the Weyl constants between rounds.                                        */
/* ------------------------------------------------------------------------- */
void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A word's top 23 bits as an odd multiple of 2^-24: exact in FP32 and FP64, */
/* strictly inside (0, 1).                                                   */
static double unit_uniform(uint32_t w)
{
    return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

static double nig_mu(const oracle_model *m)
{
    if (!isnan(m->mu)) return m->mu;
    double gam = sqrt(m->alpha * m->alpha - m->beta * m->beta);
    return -m->dbar * m->beta / gam; /* E[H_1] = mu + dbar*beta/gamma = 0 */
}

/* One driver increment Delta H over a step of length h, for (path, step).   */
/* Counter (k, inst, path_lo, path_hi), key (seed_lo, seed_hi).  Box-Muller  */
/* gives z1 (chi-square source of the IG draw, or the Brownian increment)    */
/* and z2 (the mixing normal).  margin = u2 - m/(m+y), the distance of the   */
/* IG acceptance test from its threshold.                                    */
static double draw_increment(const oracle_model *m, double h, uint64_t seed, uint32_t inst,
                             uint64_t path, uint32_t k, double *margin)
{
    uint32_t ctr[4] = {k, inst, (uint32_t)path, (uint32_t)(path >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    oracle_philox(ctr, key, w);
    double u0 = unit_uniform(w[0]), u1 = unit_uniform(w[1]), u2 = unit_uniform(w[2]);
    const double two_pi = 6.283185307179586476925286766559;
    double r = sqrt(-2.0 * log(u0));
    double z1 = r * cos(two_pi * u1);
    double z2 = r * sin(two_pi * u1);
    if (m->driver == 1) {
        if (margin) *margin = INFINITY;
        return sqrt(h) * z1;
    }
    double gam = sqrt(m->alpha * m->alpha - m->beta * m->beta);
    double mean = m->dbar * h / gam;        /* IG mean   */
    double shape = (m->dbar * h) * (m->dbar * h); /* IG shape  */
    double nu = z1 * z1;
    double ypl = mean + mean * mean * nu / (2.0 * shape) +
                 mean / (2.0 * shape) * sqrt(4.0 * mean * shape * nu + mean * mean * nu * nu);
    double y = mean * mean / ypl; /* smaller root of the MSH quadratic */
    double p = mean / (mean + y);
    double V = (u2 <= p) ? y : ypl;
    if (margin) *margin = u2 - p;
    return nig_mu(m) * h + m->beta * V + sqrt(V) * z2;
}

/* ------------------------------------------------------------------------- */
/* Model-level precomputation shared by all paths of one call.               */
/* ------------------------------------------------------------------------- */
typedef struct {
    const oracle_model *m;
    int n, S;       /* rates, steps */
    double h, c, BN;
    double *E;      /* [S][n][Q]: exp(lambda_l(t_k) x_j) - 1 */
    double *b0;     /* [S][n]: drift at the initial curve */
    double *D0;     /* [S+1][n]: sum_{m<k} b0 h */
    double *Z0;     /* [n] */
} oracle_pre;

/* Drift b(t_k, T_i) of Eq. (LIBOR-drift-PT) for weights w[l-1] = delta L_l /  */
/* (1 + delta L_l): continuous part plus the jump integral of                 */
/* (e^{lambda_i x} - 1) prod_{l>i} (1 + w_l (e^{lambda_l x} - 1)) - lambda_i x. */
static double drift_at(const oracle_pre *P, int k, int i, const double *w)
{
    const oracle_model *m = P->m;
    int n = P->n, Q = m->Q;
    const double *lamk = m->lam + (size_t)k * n;
    double li = lamk[i - 1];
    double b = 0.0;
    if (P->c != 0.0) {
        double sum = 0.0;
        for (int l = i + 1; l <= n; ++l) sum += w[l - 1] * lamk[l - 1];
        b += -0.5 * li * li * P->c - P->c * li * sum;
    }
    double A = 0.0;
    const double *Ek = P->E + (size_t)k * n * Q;
    for (int j = 0; j < Q; ++j) {
        double prod = 1.0;
        for (int l = i + 1; l <= n; ++l) prod *= 1.0 + w[l - 1] * Ek[(size_t)(l - 1) * Q + j];
        double xj = m->x[j];
        A += m->W[j] / (xj * xj) * (Ek[(size_t)(i - 1) * Q + j] * prod - li * xj);
    }
    return b - A;
}

static int pre_init(oracle_pre *P, const oracle_model *m)
{
    memset(P, 0, sizeof(*P));
    P->m = m;
    P->n = m->N - 1;
    P->S = P->n * m->s;
    P->h = m->delta / m->s;
    P->c = (m->driver == 1) ? 1.0 : 0.0;
    int n = P->n, S = P->S, Q = m->Q;
    P->E = (double *)malloc(sizeof(double) * ((size_t)S * n * (Q > 0 ? Q : 1)));
    P->b0 = (double *)malloc(sizeof(double) * (size_t)S * n);
    P->D0 = (double *)malloc(sizeof(double) * (size_t)(S + 1) * n);
    P->Z0 = (double *)malloc(sizeof(double) * n);
    double *w0 = (double *)malloc(sizeof(double) * n);
    if (!P->E || !P->b0 || !P->D0 || !P->Z0 || !w0) { free(w0); return -1; }
    for (int k = 0; k < S; ++k)
        for (int l = 0; l < n; ++l)
            for (int j = 0; j < Q; ++j)
                P->E[((size_t)k * n + l) * Q + j] = expm1(m->lam[(size_t)k * n + l] * m->x[j]);
    double BN = 1.0;
    for (int q = 0; q < m->N; ++q) BN /= 1.0 + m->delta * m->L0[q]; /* Eq. (i-val) inverted */
    P->BN = BN;
    for (int l = 1; l <= n; ++l) {
        P->Z0[l - 1] = log(m->L0[l]);
        w0[l - 1] = m->delta * m->L0[l] / (1.0 + m->delta * m->L0[l]);
    }
    /* Eq. (Picard-2): drift at Z^(0) = Z(0), then its running integral. */
    for (int k = 0; k < S; ++k)
        for (int l = 1; l <= n; ++l) P->b0[(size_t)k * n + l - 1] = drift_at(P, k, l, w0);
    for (int l = 0; l < n; ++l) P->D0[l] = 0.0;
    for (int k = 0; k < S; ++k)
        for (int l = 0; l < n; ++l)
            P->D0[(size_t)(k + 1) * n + l] = P->D0[(size_t)k * n + l] + P->b0[(size_t)k * n + l] * P->h;
    free(w0);
    return 0;
}

static void pre_free(oracle_pre *P)
{
    free(P->E); free(P->b0); free(P->D0); free(P->Z0);
}

/* ------------------------------------------------------------------------- */
/* One path of one scheme.                                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    const oracle_pre *P;
    int scheme, ns;
    uint64_t seed, path0, npaths;
    const uint64_t *plist; /* explicit path indices, or NULL for path0 + p */
    uint32_t inst;
    const double *strikes; /* [n][ns] */
    double *sum, *sumsq;   /* [n][ns], thread-local */
    double *snap;          /* [npaths][n][n] or NULL */
    double *min_margin;    /* [npaths] or NULL */
    int status;
} oracle_job;

static void run_path(oracle_job *J, uint64_t p, double *Z, double *Y, double *w, double *b)
{
    const oracle_pre *P = J->P;
    const oracle_model *m = P->m;
    int n = P->n, s = m->s, S = P->S;
    double h = P->h, delta = m->delta;
    uint64_t path = J->plist ? J->plist[p] : J->path0 + p;
    double mmin = INFINITY;
    for (int l = 0; l < n; ++l) { Z[l] = P->Z0[l]; Y[l] = 0.0; }
    for (int k = 0; k < S; ++k) {
        double margin;
        double dH = draw_increment(m, h, J->seed, J->inst, path, (uint32_t)k, &margin);
        if (margin < 0) margin = -margin;
        if (margin < mmin) mmin = margin;
        int imin = k / s + 1; /* rate i is live while k < i*s */
        const double *lamk = m->lam + (size_t)k * n;
        if (J->scheme == ORACLE_FROZEN) {
            for (int i = imin; i <= n; ++i) b[i - 1] = P->b0[(size_t)k * n + i - 1];
        } else {
            for (int l = imin; l <= n; ++l) {
                double zl = (J->scheme == ORACLE_PICARD)
                                ? P->Z0[l - 1] + P->D0[(size_t)k * n + l - 1] + Y[l - 1] /* Z^(1)(t_k) */
                                : Z[l - 1];
                double L = exp(zl);
                w[l - 1] = delta * L / (1.0 + delta * L);
            }
            for (int i = imin; i <= n; ++i) b[i - 1] = drift_at(P, k, i, w);
        }
        for (int i = imin; i <= n; ++i) {
            Z[i - 1] += b[i - 1] * h + lamk[i - 1] * dH;
            Y[i - 1] += lamk[i - 1] * dH;
        }
        if ((k + 1) % s == 0) { /* t_{k+1} = T_mat: rate mat fixes */
            int mat = (k + 1) / s;
            double num = 1.0;
            for (int l = mat + 1; l <= n; ++l) num *= 1.0 + delta * exp(Z[l - 1]);
            double Lm = exp(Z[mat - 1]);
            for (int q = 0; q < J->ns; ++q) {
                double K = J->strikes[(size_t)(mat - 1) * J->ns + q];
                double pay = delta * P->BN * num * (Lm > K ? Lm - K : 0.0);
                J->sum[(size_t)(mat - 1) * J->ns + q] += pay;
                J->sumsq[(size_t)(mat - 1) * J->ns + q] += pay * pay;
            }
            if (J->snap) {
                double *row = J->snap + ((size_t)p * n + (mat - 1)) * n;
                for (int l = 1; l <= n; ++l) row[l - 1] = (l >= mat) ? Z[l - 1] : NAN;
            }
        }
    }
    if (J->min_margin) J->min_margin[p] = mmin;
}

static void *run_job(void *arg)
{
    oracle_job *J = (oracle_job *)arg;
    int n = J->P->n;
    double *buf = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    if (!buf) { J->status = -1; return NULL; }
    for (uint64_t p = 0; p < J->npaths; ++p) run_path(J, p, buf, buf + n, buf + 2 * n, buf + 3 * n);
    free(buf);
    return NULL;
}

/* Simulate paths [path0, path0 + npaths) of one scheme.  Sums of payoffs and */
/* of squared payoffs per (maturity, strike) are accumulated per thread over */
/* contiguous path blocks and merged in thread order.                        */
static int simulate_impl(const oracle_model *m, int scheme, uint64_t seed, uint32_t inst,
                         uint64_t path0, const uint64_t *plist, uint64_t npaths, int ns,
                         const double *strikes, double *sum, double *sumsq, double *snap,
                         double *min_margin, int nthreads)
{
    if (!m || m->N < 2 || m->s < 1 || m->Q < 0 || !(m->delta > 0)) return -1;
    if (scheme != ORACLE_FULL && scheme != ORACLE_PICARD && scheme != ORACLE_FROZEN) return -1;
    oracle_pre P;
    if (pre_init(&P, m)) { pre_free(&P); return -2; }
    int n = P.n;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > npaths) nthreads = npaths > 0 ? (int)npaths : 1;
    oracle_job *jobs = (oracle_job *)calloc(nthreads, sizeof(oracle_job));
    pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
    double *acc = (double *)calloc((size_t)2 * nthreads * n * (ns > 0 ? ns : 1), sizeof(double));
    if (!jobs || !th || !acc) { free(jobs); free(th); free(acc); pre_free(&P); return -2; }
    uint64_t per = npaths / nthreads, extra = npaths % nthreads, start = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t cnt = per + ((uint64_t)t < extra ? 1 : 0);
        oracle_job *J = &jobs[t];
        J->P = &P; J->scheme = scheme; J->ns = ns; J->seed = seed; J->inst = inst;
        J->path0 = path0 + start; J->npaths = cnt; J->strikes = strikes;
        J->plist = plist ? plist + start : NULL;
        J->sum = acc + (size_t)2 * t * n * ns;
        J->sumsq = J->sum + (size_t)n * ns;
        J->snap = snap ? snap + (size_t)start * n * n : NULL;
        J->min_margin = min_margin ? min_margin + start : NULL;
        start += cnt;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    run_job(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    int status = 0;
    for (int q = 0; q < n * ns; ++q) { sum[q] = 0.0; sumsq[q] = 0.0; }
    for (int t = 0; t < nthreads; ++t) {
        if (jobs[t].status) status = jobs[t].status;
        for (int q = 0; q < n * ns; ++q) { sum[q] += jobs[t].sum[q]; sumsq[q] += jobs[t].sumsq[q]; }
    }
    free(jobs); free(th); free(acc);
    pre_free(&P);
    return status;
}

int oracle_simulate(const oracle_model *m, int scheme, uint64_t seed, uint32_t inst,
                    uint64_t path0, uint64_t npaths, int ns, const double *strikes,
                    double *sum, double *sumsq, double *snap, double *min_margin, int nthreads)
{
    return simulate_impl(m, scheme, seed, inst, path0, NULL, npaths, ns, strikes, sum, sumsq, snap,
                         min_margin, nthreads);
}

/* Same, for an explicit list of path indices (sampled paths of a large run). */
int oracle_simulate_list(const oracle_model *m, int scheme, uint64_t seed, uint32_t inst,
                         const uint64_t *paths, uint64_t npaths, int ns, const double *strikes,
                         double *sum, double *sumsq, double *snap, double *min_margin, int nthreads)
{
    return simulate_impl(m, scheme, seed, inst, 0, paths, npaths, ns, strikes, sum, sumsq, snap,
                         min_margin, nthreads);
}

/* Driver increments for paths [path0, path0+npaths) and all n*s steps:     */
/* dH[p][k] and the acceptance margins.                                      */
int oracle_increments(const oracle_model *m, uint64_t seed, uint32_t inst, uint64_t path0,
                      uint64_t npaths, double *dH, double *margin)
{
    if (!m || m->N < 2 || m->s < 1) return -1;
    int S = (m->N - 1) * m->s;
    double h = m->delta / m->s;
    for (uint64_t p = 0; p < npaths; ++p)
        for (int k = 0; k < S; ++k) {
            double mg;
            dH[p * S + k] = draw_increment(m, h, seed, inst, path0 + p, (uint32_t)k, &mg);
            if (margin) margin[p * S + k] = mg;
        }
    return 0;
}

/* Drift b(t_k, T_i) for caller weights w[l-1], l = 1..n. */
int oracle_drift(const oracle_model *m, int k, int i, const double *w, double *b)
{
    if (!m || m->N < 2) return -1;
    int n = m->N - 1;
    if (k < 0 || k >= n * m->s || i < 1 || i > n) return -1;
    oracle_pre P;
    if (pre_init(&P, m)) { pre_free(&P); return -2; }
    *b = drift_at(&P, k, i, w);
    pre_free(&P);
    return 0;
}

/* Frozen-curve drift b0[k][l-1] and its running integral D0[k][l-1]. */
int oracle_frozen_drift(const oracle_model *m, double *b0, double *D0)
{
    if (!m || m->N < 2 || m->s < 1) return -1;
    oracle_pre P;
    if (pre_init(&P, m)) { pre_free(&P); return -2; }
    int n = P.n, S = P.S;
    memcpy(b0, P.b0, sizeof(double) * (size_t)S * n);
    memcpy(D0, P.D0, sizeof(double) * (size_t)(S + 1) * n);
    pre_free(&P);
    return 0;
}
