/*
 * lbm_oracle.c -- FP64 CPU oracle for the Galilean-invariant filtered lattice
 * Boltzmann collision of Chen, Zhang & Gopalakrishnan (arXiv 2002.02503).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, literal statement of
 * the method that the CUDA library is checked against.  Only the test suite,
 * the package's smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes, in the paper's order and notation (lattice units, dx=dt=1):
 *   1. rho = sum_i f_i,  rho u = sum_i c_i f_i                        (Eq. mme)
 *   2. f^eq_i = w_i rho sum_{n=0}^{K} H^(n)(xi_i) : V^[n] / n!        (Eq. hermite,
 *      truncated at n <= K as the isotropy argument of Sec. 2 and Sec. 3 asks),
 *      with xi_i = c_i / sqrt(T0), V = u / sqrt(T0)
 *   3. f^neq_i = f_i - f^eq_i                                         (Eq. neq)
 *   4. Pi^neq = sum_i (c_i - u)(c_i - u) f^neq_i                      (Eq. Pi_def,
 *      the relative-frame definition)
 *   5. fhat^neq_i = w_i/(2 T0) sum_{n=2}^{K} H^(n)(xi_i) : V^[n-2] Pi^neq / (n-2)!
 *                                                                     (Eq. hermite-coll)
 *   6. f'_i = f^eq_i + (1 - 1/tau) fhat^neq_i                         (Eq. post-1 with
 *      the filtered non-equilibrium part, i.e. Eq. lbe-reg)
 *   7. f_i(x + c_i, t+1) = f'_i(x, t), periodic                        (Eq. lbe, push form)
 * The tensor Hermite polynomials H^(n)(xi) are built generically by the
 * recursion of Eq. recurG (Appendix), H^(0)=1, H^(1)_a = xi_a.
 *
 * Energy-flux extension (Sec. 4, Eq. pq): fhat^neq = fhat^{neq,p} + theta fhat^{neq,q} with
 *   Qt^neq = sum_i c'_i c'_i c'_i f^neq_i                                (Eq. Q_def)
 *   fhat^{neq,q}_i = w_i/(6 T0^{3/2}) sum_{n=3}^{K} H^(n)(xi_i) : V^[n-3] Qt^neq / (n-3)!
 * the Hermite series of the compact Eq. filter-Q (read with the 1/rho of Eq. filter-coll),
 * obtained from the generating function of the H^(n) exactly as the Appendix obtains
 * Eq. hermite-coll, one derivative higher; truncated at the same order K.
 *
 * Lattice tables: the paper fixes T0 = 1/3 for D3Q15/D3Q19 (Sec. 2, after
 * Eq. iso) and the isotropy classes 2N (D2Q9, D3Q15, D3Q19: 4; D3Q39: 6), but prints
 * no weights.  The standard velocity sets below are used; the test suite checks
 * them against the isotropy identities of Eq. iso.  D3Q27 is not in the paper;
 * it is the standard 27-velocity set (isotropy class 4).
 *
 * Build: gcc -O2 -fPIC -shared -pthread lbm_oracle.c -o liblbm_oracle.so -lm
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXQ 39
#define ORC_MAX_K 10 /* highest Hermite order the oracle builds (3^10 tensor entries) */

enum { ORC_D2Q9 = 0, ORC_D3Q19 = 1, ORC_D3Q27 = 2, ORC_D3Q39 = 3, ORC_D3Q15 = 4 };

typedef struct {
    int D, Q;
    double T0;
    int c[ORC_MAXQ][3];
    double w[ORC_MAXQ];
} orc_lattice_t;

/* ---------------------------------------------------------------- tables */

/* Append every distinct vector obtained from (a,b,c) by permuting the
 * components and flipping signs (restricted to the first D components). */
static void add_shell(orc_lattice_t *L, int D, int a, int b, int c, double w) {
    int base[3] = {a, b, c};
    static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int p = 0; p < 6; ++p) {
        for (int s = 0; s < 8; ++s) {
            int v[3];
            for (int k = 0; k < 3; ++k) {
                v[k] = base[perm[p][k]];
                if (s & (1 << k)) v[k] = -v[k];
            }
            if (D == 2 && v[2] != 0) continue;
            int dup = 0;
            for (int q = 0; q < L->Q && !dup; ++q)
                if (L->c[q][0] == v[0] && L->c[q][1] == v[1] && L->c[q][2] == v[2]) dup = 1;
            if (dup) continue;
            L->c[L->Q][0] = v[0];
            L->c[L->Q][1] = v[1];
            L->c[L->Q][2] = v[2];
            L->w[L->Q] = w;
            L->Q++;
        }
    }
}

static int make_lattice(int lat, orc_lattice_t *L) {
    memset(L, 0, sizeof(*L));
    switch (lat) {
    case ORC_D2Q9: /* w = 4/9, 1/9, 1/36; T0 = 1/3 */
        L->D = 2;
        L->T0 = 1.0 / 3.0;
        add_shell(L, 2, 0, 0, 0, 4.0 / 9.0);
        add_shell(L, 2, 1, 0, 0, 1.0 / 9.0);
        add_shell(L, 2, 1, 1, 0, 1.0 / 36.0);
        break;
    case ORC_D3Q15: /* w = 2/9, 1/9, 1/72; T0 = 1/3 */
        L->D = 3;
        L->T0 = 1.0 / 3.0;
        add_shell(L, 3, 0, 0, 0, 2.0 / 9.0);
        add_shell(L, 3, 1, 0, 0, 1.0 / 9.0);
        add_shell(L, 3, 1, 1, 1, 1.0 / 72.0);
        break;
    case ORC_D3Q19: /* w = 1/3, 1/18, 1/36; T0 = 1/3 */
        L->D = 3;
        L->T0 = 1.0 / 3.0;
        add_shell(L, 3, 0, 0, 0, 1.0 / 3.0);
        add_shell(L, 3, 1, 0, 0, 1.0 / 18.0);
        add_shell(L, 3, 1, 1, 0, 1.0 / 36.0);
        break;
    case ORC_D3Q27: /* w = 8/27, 2/27, 1/54, 1/216; T0 = 1/3 */
        L->D = 3;
        L->T0 = 1.0 / 3.0;
        add_shell(L, 3, 0, 0, 0, 8.0 / 27.0);
        add_shell(L, 3, 1, 0, 0, 2.0 / 27.0);
        add_shell(L, 3, 1, 1, 0, 1.0 / 54.0);
        add_shell(L, 3, 1, 1, 1, 1.0 / 216.0);
        break;
    case ORC_D3Q39: /* six shells; T0 = 2/3 */
        L->D = 3;
        L->T0 = 2.0 / 3.0;
        add_shell(L, 3, 0, 0, 0, 1.0 / 12.0);
        add_shell(L, 3, 1, 0, 0, 1.0 / 12.0);
        add_shell(L, 3, 1, 1, 1, 1.0 / 27.0);
        add_shell(L, 3, 2, 0, 0, 2.0 / 135.0);
        add_shell(L, 3, 2, 2, 0, 1.0 / 432.0);
        add_shell(L, 3, 3, 0, 0, 1.0 / 1620.0);
        break;
    default:
        return -1;
    }
    return 0;
}

/* ------------------------------------------------- Hermite tensors, Eq. recurG
 * A rank-n tensor over D components is stored densely as D^n doubles; the
 * multi-index (a_1..a_n) has flat index sum_k a_k D^(n-k) (a_1 most significant). */

static long ipow(int b, int e) {
    long r = 1;
    while (e-- > 0) r *= b;
    return r;
}

typedef struct {
    int D, K;
    double *H[ORC_MAX_K + 1]; /* H[n] has D^n entries */
} orc_hermite_t;

/* Build H^(0..K)(xi) for one velocity by Eq. recurG:
 *   H^(n+1)_{a1..a(n+1)} = xi_{a(n+1)} H^(n)_{a1..an}
 *                          - sum_{k=1}^{n} delta_{a(n+1) ak} H^(n-1)_{a1..(ak omitted)..an} */
static int hermite_build(int D, int K, const double *xi, orc_hermite_t *h) {
    h->D = D;
    h->K = K;
    for (int n = 0; n <= K; ++n) {
        h->H[n] = (double *)calloc((size_t)ipow(D, n), sizeof(double));
        if (!h->H[n]) return -1;
    }
    h->H[0][0] = 1.0;
    if (K >= 1)
        for (int a = 0; a < D; ++a) h->H[1][a] = xi[a];
    int digits[ORC_MAX_K + 1];
    for (int n = 1; n < K; ++n) { /* build H^(n+1) from H^(n), H^(n-1) */
        long size = ipow(D, n + 1);
        for (long idx = 0; idx < size; ++idx) {
            long t = idx;
            for (int k = n; k >= 0; --k) { /* digits[0]=a1 ... digits[n]=a(n+1) */
                digits[k] = (int)(t % D);
                t /= D;
            }
            int last = digits[n];
            double v = xi[last] * h->H[n][idx / D];
            for (int k = 0; k < n; ++k) {
                if (digits[k] != last) continue;
                long red = 0; /* flat index of a1..an with a_k removed (rank n-1) */
                for (int m = 0; m < n; ++m)
                    if (m != k) red = red * D + digits[m];
                v -= h->H[n - 1][red];
            }
            h->H[n + 1][idx] = v;
        }
    }
    return 0;
}

static void hermite_free(orc_hermite_t *h) {
    for (int n = 0; n <= h->K; ++n) free(h->H[n]);
}

/* Per-lattice context: tables plus H^(n)(xi_i) for every velocity. */
typedef struct {
    orc_lattice_t L;
    int K;
    orc_hermite_t herm[ORC_MAXQ];
} orc_ctx_t;

static void ctx_free(orc_ctx_t *ctx) {
    for (int i = 0; i < ctx->L.Q; ++i) hermite_free(&ctx->herm[i]);
}

static int ctx_init(int lat, int K, orc_ctx_t *ctx) {
    memset(ctx, 0, sizeof(*ctx));
    if (K < 0 || K > ORC_MAX_K) return -2;
    if (make_lattice(lat, &ctx->L)) return -1;
    ctx->K = K;
    double s = 1.0 / sqrt(ctx->L.T0);
    for (int i = 0; i < ctx->L.Q; ++i) {
        double xi[3];
        for (int a = 0; a < 3; ++a) xi[a] = ctx->L.c[i][a] * s;
        if (hermite_build(ctx->L.D, K, xi, &ctx->herm[i])) {
            ctx_free(ctx);
            return -3;
        }
    }
    return 0;
}

/* ------------------------------------------------------ per-cell operations */

static double factorial(int n) {
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= k;
    return r;
}

/* Work space for the products V^[n] and V^[n-2] Pi, one per thread. */
typedef struct {
    double *Vp[ORC_MAX_K + 1]; /* V^[n], D^n entries */
    double *VPi[ORC_MAX_K + 1]; /* V^[n-2] (x) Pi, D^n entries (n >= 2); reused for V^[n-3] (x) Qt */
    int D, K;
} orc_work_t;

static int work_init(int D, int K, orc_work_t *wk) {
    memset(wk, 0, sizeof(*wk));
    wk->D = D;
    wk->K = K;
    for (int n = 0; n <= K; ++n) {
        wk->Vp[n] = (double *)calloc((size_t)ipow(D, n), sizeof(double));
        wk->VPi[n] = (double *)calloc((size_t)ipow(D, n), sizeof(double));
        if (!wk->Vp[n] || !wk->VPi[n]) return -1;
    }
    return 0;
}

static void work_free(orc_work_t *wk) {
    for (int n = 0; n <= wk->K; ++n) {
        free(wk->Vp[n]);
        free(wk->VPi[n]);
    }
}

static void fill_Vpowers(orc_work_t *wk, const double *V) {
    int D = wk->D;
    wk->Vp[0][0] = 1.0;
    for (int n = 0; n < wk->K; ++n) {
        long size = ipow(D, n);
        for (long p = 0; p < size; ++p)
            for (int a = 0; a < D; ++a) wk->Vp[n + 1][p * D + a] = wk->Vp[n][p] * V[a];
    }
}

/* f^eq_i = w_i rho sum_{n=0}^{K} H^(n)(xi_i) : V^[n] / n!   (Eq. hermite, truncated) */
static void feq_cell(const orc_ctx_t *ctx, orc_work_t *wk, double rho, const double *u, double *feq) {
    const orc_lattice_t *L = &ctx->L;
    double s = 1.0 / sqrt(L->T0);
    double V[3] = {u[0] * s, u[1] * s, u[2] * s};
    fill_Vpowers(wk, V);
    for (int i = 0; i < L->Q; ++i) {
        double sum = 0.0;
        for (int n = 0; n <= ctx->K; ++n) {
            long size = ipow(L->D, n);
            double dot = 0.0;
            for (long k = 0; k < size; ++k) dot += ctx->herm[i].H[n][k] * wk->Vp[n][k];
            sum += dot / factorial(n);
        }
        feq[i] = L->w[i] * rho * sum;
    }
}

/* fhat^neq_i = w_i/(2 T0) sum_{n=2}^{K} H^(n)(xi_i) : V^[n-2] Pi / (n-2)!   (Eq. hermite-coll)
 * Pi is a full D x D matrix stored row-major in a 3x3 array. */
static void fneq_hat_cell(const orc_ctx_t *ctx, orc_work_t *wk, const double *u, const double Pi[3][3],
                          double *fhat) {
    const orc_lattice_t *L = &ctx->L;
    int D = L->D;
    double s = 1.0 / sqrt(L->T0);
    double V[3] = {u[0] * s, u[1] * s, u[2] * s};
    fill_Vpowers(wk, V);
    for (int n = 2; n <= ctx->K; ++n) {
        long size = ipow(D, n);
        for (long idx = 0; idx < size; ++idx) {
            int g = (int)(idx % D);
            int b = (int)((idx / D) % D);
            wk->VPi[n][idx] = wk->Vp[n - 2][idx / (D * D)] * Pi[b][g];
        }
    }
    for (int i = 0; i < L->Q; ++i) {
        double sum = 0.0;
        for (int n = 2; n <= ctx->K; ++n) {
            long size = ipow(D, n);
            double dot = 0.0;
            for (long k = 0; k < size; ++k) dot += ctx->herm[i].H[n][k] * wk->VPi[n][k];
            sum += dot / factorial(n - 2);
        }
        fhat[i] = L->w[i] / (2.0 * L->T0) * sum;
    }
}

/* fhat^{neq,q}_i = w_i/(6 T0^{3/2}) sum_{n=3}^{K} H^(n)(xi_i) : V^[n-3] Qt / (n-3)!
 * Qt is a full D x D x D tensor stored in a 3x3x3 array. */
static void fneq_hat_q_cell(const orc_ctx_t *ctx, orc_work_t *wk, const double *u, const double Qt[3][3][3],
                            double *out) {
    const orc_lattice_t *L = &ctx->L;
    int D = L->D;
    double s = 1.0 / sqrt(L->T0);
    double V[3] = {u[0] * s, u[1] * s, u[2] * s};
    fill_Vpowers(wk, V);
    for (int n = 3; n <= ctx->K; ++n) {
        long size = ipow(D, n);
        for (long idx = 0; idx < size; ++idx) {
            int c3 = (int)(idx % D);
            int c2 = (int)((idx / D) % D);
            int c1 = (int)((idx / (D * D)) % D);
            wk->VPi[n][idx] = wk->Vp[n - 3][idx / (D * D * D)] * Qt[c1][c2][c3];
        }
    }
    for (int i = 0; i < L->Q; ++i) {
        double sum = 0.0;
        for (int n = 3; n <= ctx->K; ++n) {
            long size = ipow(D, n);
            double dot = 0.0;
            for (long k = 0; k < size; ++k) dot += ctx->herm[i].H[n][k] * wk->VPi[n][k];
            sum += dot / factorial(n - 3);
        }
        out[i] = L->w[i] / (6.0 * L->T0 * sqrt(L->T0)) * sum;
    }
}

/* Eq. mme */
static void moments_cell(const orc_lattice_t *L, const double *f, double *rho, double *u) {
    double r = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < L->Q; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) j[a] += L->c[i][a] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

/* Collision models: the paper's filtered collision (Eq. lbe-reg), or the BGK
 * operator of Eq. BGK, C_i = -(f_i - f^eq_i)/tau, with the same truncated f^eq --
 * the unfiltered baseline the paper compares against in Sec. 1 and Sec. 4. */
enum { ORC_FILTERED = 0, ORC_BGK = 1 };

/* One cell through steps 1-6 of the header.  Intermediates are returned when
 * the pointers are non-NULL. */
static void collide_cell_model(const orc_ctx_t *ctx, orc_work_t *wk, double tau, int model, double theta,
                               const double *f, double *fpost, double *rho_out, double *u_out, double *feq_out,
                               double *Pi_out, double *fhat_out, double *Qt_out, double *fhatq_out);

static void collide_cell(const orc_ctx_t *ctx, orc_work_t *wk, double tau, const double *f, double *fpost,
                         double *rho_out, double *u_out, double *feq_out, double *Pi_out, double *fhat_out) {
    collide_cell_model(ctx, wk, tau, ORC_FILTERED, 0.0, f, fpost, rho_out, u_out, feq_out, Pi_out, fhat_out, NULL,
                       NULL);
}

static void collide_cell_model(const orc_ctx_t *ctx, orc_work_t *wk, double tau, int model, double theta,
                               const double *f, double *fpost, double *rho_out, double *u_out, double *feq_out,
                               double *Pi_out, double *fhat_out, double *Qt_out, double *fhatq_out) {
    const orc_lattice_t *L = &ctx->L;
    double rho, u[3], feq[ORC_MAXQ], fneq[ORC_MAXQ], fhat[ORC_MAXQ];
    moments_cell(L, f, &rho, u);
    feq_cell(ctx, wk, rho, u, feq);
    for (int i = 0; i < L->Q; ++i) fneq[i] = f[i] - feq[i];
    double Pi[3][3] = {{0}};
    for (int i = 0; i < L->Q; ++i) { /* Eq. Pi_def: relative velocity c' = c - u */
        double cr[3];
        for (int a = 0; a < 3; ++a) cr[a] = L->c[i][a] - u[a];
        for (int a = 0; a < L->D; ++a)
            for (int b = 0; b < L->D; ++b) Pi[a][b] += cr[a] * cr[b] * fneq[i];
    }
    fneq_hat_cell(ctx, wk, u, (const double(*)[3])Pi, fhat);
    double fhq[ORC_MAXQ] = {0};
    double Qt[3][3][3] = {{{0}}};
    if (theta != 0.0 || Qt_out || fhatq_out) {
        for (int i = 0; i < L->Q; ++i) { /* Eq. Q_def: relative velocity c' = c - u */
            double cr[3];
            for (int a = 0; a < 3; ++a) cr[a] = L->c[i][a] - u[a];
            for (int a = 0; a < L->D; ++a)
                for (int b = 0; b < L->D; ++b)
                    for (int c = 0; c < L->D; ++c) Qt[a][b][c] += cr[a] * cr[b] * cr[c] * fneq[i];
        }
        fneq_hat_q_cell(ctx, wk, u, (const double(*)[3][3])Qt, fhq);
    }
    double relax = 1.0 - 1.0 / tau;
    if (model == ORC_BGK) /* Eq. BGK: f' = f - (f - f^eq)/tau */
        for (int i = 0; i < L->Q; ++i) fpost[i] = f[i] - (f[i] - feq[i]) / tau;
    else /* Eq. lbe-reg with Eq. pq: fhat = fhat^p + theta fhat^q */
        for (int i = 0; i < L->Q; ++i) fpost[i] = feq[i] + relax * (fhat[i] + theta * fhq[i]);
    if (Qt_out)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c) Qt_out[9 * a + 3 * b + c] = Qt[a][b][c];
    if (fhatq_out) memcpy(fhatq_out, fhq, sizeof(double) * L->Q);
    if (rho_out) *rho_out = rho;
    if (u_out)
        for (int a = 0; a < 3; ++a) u_out[a] = u[a];
    if (feq_out) memcpy(feq_out, feq, sizeof(double) * L->Q);
    if (fhat_out) memcpy(fhat_out, fhat, sizeof(double) * L->Q);
    if (Pi_out)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Pi_out[3 * a + b] = Pi[a][b];
}

/* ------------------------------------------------------ grid operations
 * Distributions are SoA: f[i * C + cell], cell = x + nx (y + ny z), C = nx ny nz.
 * Velocity i is the oracle's own ordering (orc_lattice reports it). */

static long wrap(long v, long n) {
    v %= n;
    return v < 0 ? v + n : v;
}

typedef struct {
    const orc_ctx_t *ctx;
    double tau;
    int model;
    double theta;
    long nx, ny, nz;
    const double *f;
    double *fnew;
    long r0, r1; /* rows (y + ny z) handled by this thread */
    int err;
} step_job_t;

static void *step_worker(void *arg) {
    step_job_t *job = (step_job_t *)arg;
    const orc_lattice_t *L = &job->ctx->L;
    long C = job->nx * job->ny * job->nz;
    orc_work_t wk;
    if (work_init(L->D, job->ctx->K, &wk)) {
        job->err = -1;
        work_free(&wk);
        return NULL;
    }
    double fc[ORC_MAXQ], fp[ORC_MAXQ];
    for (long r = job->r0; r < job->r1; ++r) {
        const long y = r % job->ny, z = r / job->ny;
        for (long x = 0; x < job->nx; ++x) {
                long cell = x + job->nx * (y + job->ny * z);
                for (int i = 0; i < L->Q; ++i) fc[i] = job->f[i * C + cell];
                collide_cell_model(job->ctx, &wk, job->tau, job->model, job->theta, fc, fp, NULL, NULL, NULL, NULL,
                                   NULL, NULL, NULL);
                for (int i = 0; i < L->Q; ++i) { /* Eq. lbe: push to x + c_i */
                    long xd = wrap(x + L->c[i][0], job->nx);
                    long yd = wrap(y + L->c[i][1], job->ny);
                    long zd = wrap(z + L->c[i][2], job->nz);
                    job->fnew[i * C + xd + job->nx * (yd + job->ny * zd)] = fp[i];
                }
            }
    }
    work_free(&wk);
    return NULL;
}

static int run_parallel(const orc_ctx_t *ctx, double tau, int model, double theta, const int64_t *dims,
                        const double *f, double *fnew, int nthreads) {
    long rows = dims[1] * dims[2];
    if (nthreads < 1) nthreads = 1;
    if (nthreads > rows) nthreads = (int)rows;
    step_job_t jobs[256];
    pthread_t th[256];
    if (nthreads > 256) nthreads = 256;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].ctx = ctx;
        jobs[t].tau = tau;
        jobs[t].model = model;
        jobs[t].theta = theta;
        jobs[t].nx = dims[0];
        jobs[t].ny = dims[1];
        jobs[t].nz = dims[2];
        jobs[t].f = f;
        jobs[t].fnew = fnew;
        jobs[t].r0 = rows * t / nthreads;
        jobs[t].r1 = rows * (t + 1) / nthreads;
        jobs[t].err = 0;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, step_worker, &jobs[t]);
    step_worker(&jobs[0]);
    int err = jobs[0].err;
    for (int t = 1; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].err) err = jobs[t].err;
    }
    return err;
}

static int dims_ok(const orc_lattice_t *L, const int64_t *dims) {
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return 0;
    if (L->D == 2 && dims[2] != 1) return 0;
    return 1;
}

/* ------------------------------------------------------ exported C API
 * Every function returns 0 on success and a negative code on bad arguments. */

int orc_lattice(int lat, int *D, int *Q, double *T0, int *c /* [Q][3] */, double *w /* [Q] */) {
    orc_lattice_t L;
    if (make_lattice(lat, &L)) return -1;
    if (D) *D = L.D;
    if (Q) *Q = L.Q;
    if (T0) *T0 = L.T0;
    for (int i = 0; i < L.Q; ++i) {
        if (c)
            for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
        if (w) w[i] = L.w[i];
    }
    return 0;
}

/* H^(n)(xi_i) for velocity i of the lattice, D^n entries. */
int orc_hermite(int lat, int i, int n, double *out) {
    orc_ctx_t ctx;
    int rc = ctx_init(lat, n < 1 ? 1 : n, &ctx);
    if (rc) return rc;
    if (i < 0 || i >= ctx.L.Q) {
        ctx_free(&ctx);
        return -4;
    }
    memcpy(out, ctx.herm[i].H[n], sizeof(double) * (size_t)ipow(ctx.L.D, n));
    ctx_free(&ctx);
    return 0;
}

int orc_feq(int lat, int K, double rho, const double *u, double *feq) {
    orc_ctx_t ctx;
    int rc = ctx_init(lat, K, &ctx);
    if (rc) return rc;
    orc_work_t wk;
    if (work_init(ctx.L.D, K, &wk)) rc = -3;
    else feq_cell(&ctx, &wk, rho, u, feq);
    work_free(&wk);
    ctx_free(&ctx);
    return rc;
}

int orc_fneq_hat(int lat, int K, const double *u, const double *Pi /* [3][3] */, double *fhat) {
    orc_ctx_t ctx;
    int rc = ctx_init(lat, K, &ctx);
    if (rc) return rc;
    orc_work_t wk;
    double P[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) P[a][b] = Pi[3 * a + b];
    if (work_init(ctx.L.D, K, &wk)) rc = -3;
    else fneq_hat_cell(&ctx, &wk, u, (const double(*)[3])P, fhat);
    work_free(&wk);
    ctx_free(&ctx);
    return rc;
}

/* One cell: f (Q) -> f' (Q) plus the intermediates of steps 1-5. */
int orc_collide(int lat, int K, double tau, const double *f, double *fpost, double *rho, double *u /* [3] */,
                double *feq, double *Pi /* [9] */, double *fhat) {
    orc_ctx_t ctx;
    int rc = ctx_init(lat, K, &ctx);
    if (rc) return rc;
    orc_work_t wk;
    if (work_init(ctx.L.D, K, &wk)) rc = -3;
    else collide_cell(&ctx, &wk, tau, f, fpost, rho, u, feq, Pi, fhat);
    work_free(&wk);
    ctx_free(&ctx);
    return rc;
}

/* f := f^eq_K(rho, u) at every cell (no non-equilibrium part).
 * rho: [C], u: [D][C] (SoA), f: [Q][C].  Cells are split over threads. */
typedef struct {
    const orc_ctx_t *ctx;
    long C, c0, c1;
    const double *rho, *u;
    double *f;
    int err;
} init_job_t;

static void *init_worker(void *arg) {
    init_job_t *job = (init_job_t *)arg;
    const orc_lattice_t *L = &job->ctx->L;
    orc_work_t wk;
    if (work_init(L->D, job->ctx->K, &wk)) {
        job->err = -3;
        work_free(&wk);
        return NULL;
    }
    double feq[ORC_MAXQ];
    for (long cell = job->c0; cell < job->c1; ++cell) {
        double uc[3] = {0, 0, 0};
        for (int a = 0; a < L->D; ++a) uc[a] = job->u[a * job->C + cell];
        feq_cell(job->ctx, &wk, job->rho[cell], uc, feq);
        for (int i = 0; i < L->Q; ++i) job->f[i * job->C + cell] = feq[i];
    }
    work_free(&wk);
    return NULL;
}

int orc_init_eq(int lat, int K, const int64_t *dims, const double *rho, const double *u, double *f, int nthreads) {
    orc_ctx_t ctx;
    int rc = ctx_init(lat, K, &ctx);
    if (rc) return rc;
    if (!dims_ok(&ctx.L, dims)) {
        ctx_free(&ctx);
        return -5;
    }
    long C = dims[0] * dims[1] * dims[2];
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > C) nthreads = (int)C;
    init_job_t jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].ctx = &ctx;
        jobs[t].C = C;
        jobs[t].c0 = C * t / nthreads;
        jobs[t].c1 = C * (t + 1) / nthreads;
        jobs[t].rho = rho;
        jobs[t].u = u;
        jobs[t].f = f;
        jobs[t].err = 0;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, init_worker, &jobs[t]);
    init_worker(&jobs[0]);
    rc = jobs[0].err;
    for (int t = 1; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].err) rc = jobs[t].err;
    }
    ctx_free(&ctx);
    return rc;
}

/* rho: [C], u: [D][C] of the distributions f: [Q][C]  (Eq. mme). */
int orc_moments(int lat, const int64_t *dims, const double *f, double *rho, double *u) {
    orc_lattice_t L;
    if (make_lattice(lat, &L)) return -1;
    if (!dims_ok(&L, dims)) return -5;
    long C = dims[0] * dims[1] * dims[2];
    double fc[ORC_MAXQ];
    for (long cell = 0; cell < C; ++cell) {
        double r, uc[3];
        for (int i = 0; i < L.Q; ++i) fc[i] = f[i * C + cell];
        moments_cell(&L, fc, &r, uc);
        rho[cell] = r;
        for (int a = 0; a < L.D; ++a) u[a * C + cell] = uc[a];
    }
    return 0;
}

/* nsteps of collide + push with the given collision model (ORC_FILTERED or ORC_BGK).
 * f holds f(t) on entry and f(t + nsteps) on exit. */
int orc_run_model(int lat, int K, double tau, int model, double theta, const int64_t *dims, double *f,
                  int64_t nsteps, int nthreads) {
    orc_ctx_t ctx;
    int rc = ctx_init(lat, K, &ctx);
    if (rc) return rc;
    if (!dims_ok(&ctx.L, dims) || nsteps < 0) {
        ctx_free(&ctx);
        return -5;
    }
    size_t n = (size_t)ctx.L.Q * (size_t)(dims[0] * dims[1] * dims[2]);
    double *tmp = (double *)malloc(n * sizeof(double));
    if (!tmp) {
        ctx_free(&ctx);
        return -3;
    }
    double *a = f, *b = tmp;
    for (int64_t s = 0; s < nsteps && rc == 0; ++s) {
        rc = run_parallel(&ctx, tau, model, theta, dims, a, b, nthreads);
        double *t = a;
        a = b;
        b = t;
    }
    if (a != f) memcpy(f, a, n * sizeof(double));
    free(tmp);
    ctx_free(&ctx);
    return rc;
}

/* nsteps of the paper's filtered collision + push. */
int orc_run(int lat, int K, double tau, const int64_t *dims, double *f, int64_t nsteps, int nthreads) {
    return orc_run_model(lat, K, tau, ORC_FILTERED, 0.0, dims, f, nsteps, nthreads);
}

/* One cell with the BGK operator (Eq. BGK) and the truncated f^eq. */
int orc_collide_bgk(int lat, int K, double tau, const double *f, double *fpost) {
    orc_ctx_t ctx;
    int rc = ctx_init(lat, K, &ctx);
    if (rc) return rc;
    orc_work_t wk;
    if (work_init(ctx.L.D, K, &wk)) rc = -3;
    else collide_cell_model(&ctx, &wk, tau, ORC_BGK, 0.0, f, fpost, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
    work_free(&wk);
    ctx_free(&ctx);
    return rc;
}

/* fhat^{neq,q} at one cell for a given Qt (Eq. pq series, truncated at K). */
int orc_fneq_hat_q(int lat, int K, const double *u, const double *Qt /* [27] */, double *out) {
    orc_ctx_t ctx;
    int rc = ctx_init(lat, K, &ctx);
    if (rc) return rc;
    orc_work_t wk;
    double T[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) T[a][b][c] = Qt[9 * a + 3 * b + c];
    if (work_init(ctx.L.D, K, &wk)) rc = -3;
    else fneq_hat_q_cell(&ctx, &wk, u, (const double(*)[3][3])T, out);
    work_free(&wk);
    ctx_free(&ctx);
    return rc;
}

/* One cell of the filtered collision with the energy-flux term (Eq. pq); returns Qt and fhat^q too. */
int orc_collide_theta(int lat, int K, double tau, double theta, const double *f, double *fpost, double *Qt,
                      double *fhatq) {
    orc_ctx_t ctx;
    int rc = ctx_init(lat, K, &ctx);
    if (rc) return rc;
    orc_work_t wk;
    if (work_init(ctx.L.D, K, &wk)) rc = -3;
    else collide_cell_model(&ctx, &wk, tau, ORC_FILTERED, theta, f, fpost, NULL, NULL, NULL, NULL, NULL, Qt, fhatq);
    work_free(&wk);
    ctx_free(&ctx);
    return rc;
}
