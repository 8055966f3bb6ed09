/*
 * FP64 CPU oracle for the exact two-dimensional DCT (test infrastructure).
 *
 * This file is test infrastructure only.  The tests, the package's smoke()
 * check and the benchmark's CPU-baseline leg may call it; the CUDA library
 * never does, and the two share no code, tables or constants.
 *
 * What it computes (BRiDCT paper, Section 2.1):
 *   Eq. 1   (Q_n)_{kj} = alpha_k cos[(pi/n)(j + 1/2) k],
 *           alpha_0 = n^{-1/2}, alpha_k = (2/n)^{1/2} for k > 0.
 *   Eq. 2   C(X) = Q_h X Q_w^T   (forward, DCT-II),
 *           C^{-1}(Y) = Q_h^T Y Q_w   (inverse, DCT-III, the adjoint).
 *   Section 7.1 gives the rectangular operator Q_h X Q_w^T for X in R^{h x w}.
 *   The round trip C^{-1}(C(X)) has exact result X (Section 2.1).
 *   Prop. 1 (Eq. 4): the transform -- diagonal spectral operator -- inverse
 *   composition U^T Lambda U, i.e. Q_h^T (Lambda o (Q_h X Q_w^T)) Q_w.
 *
 * The unnormalized convention (Section 2.1 names FFTW's REDFT10/REDFT01 pair,
 * pair factor 2n per axis) is read as
 *   forward  y_k = 2 sum_j x_j cos(pi (2j+1) k / (2n))
 *   inverse  x_j = y_0 + 2 sum_{k>=1} y_k cos(pi (2j+1) k / (2n)).
 *
 * Everything is a plain double-precision sum, applied separably (first along
 * rows, then along columns), exactly as Eq. 2 is written.  A second, brute-force
 * O(h^2 w^2) evaluation of the same double sum, with the cosine taken straight
 * from libm, serves as an independent check of the separable form.
 *
 * A planted-fault switch (oracle_set_fault) lets the CPU tests show that their
 * pins catch a dropped term, a wrong scale, a wrong index or a transposed
 * operand.  It is off (0) unless a test turns it on.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <sched.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_NORM_ORTHO 0
#define ORACLE_NORM_NONE 1

#define ORACLE_DIR_FORWARD 1
#define ORACLE_DIR_INVERSE 2

static int g_fault = 0;

/* Planted faults, for the tests of the pins only:
 *   1  alpha_0 taken as (2/n)^{1/2}                     (wrong scale)
 *   2  last term of every 1D sum dropped                (dropped term)
 *   3  cos argument uses (2j-1) instead of (2j+1)        (wrong index)
 *   4  inverse uses M instead of M^T                     (transposed operand)
 *   5  row axis uses the column-axis matrix              (swapped axes)
 *   6  spectral diagonal read as Lambda[l][k]            (transposed table) */
void oracle_set_fault(int f) { g_fault = f; }
int oracle_get_fault(void) { return g_fault; }

/* cos(pi * m / d) for integers m >= 0 and d > 0, with the argument reduced
 * exactly in integers so that the zeros and the +-1 values come out exact and
 * the remaining argument lies in [0, pi/4]. */
double oracle_cospi_frac(int64_t m, int64_t d)
{
    int64_t r = m % (2 * d);
    if (r < 0) r += 2 * d;
    if (r > d) r = 2 * d - r;            /* cos(2pi - t) = cos t, r in [0, d] */
    double sign = 1.0;
    if (2 * r > d) { r = d - r; sign = -1.0; } /* cos(pi - t) = -cos t, r in [0, d/2] */
    if (r == 0) return sign;
    if (2 * r == d) return 0.0;
    if (4 * r > d) /* cos t = sin(pi/2 - t) with pi/2 - t = pi (d - 2r) / (2d) */
        return sign * sin(M_PI * (double)(d - 2 * r) / (double)(2 * d));
    return sign * cos(M_PI * (double)r / (double)d);
}

/* Unscaled DCT-II kernel G_n[k][j] = cos(pi (2j+1) k / (2n)), row-major n x n. */
static void basis(int n, double *G)
{
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j) {
            int64_t odd = (g_fault == 3) ? (2 * (int64_t)j - 1) : (2 * (int64_t)j + 1);
            G[(size_t)k * n + j] = oracle_cospi_frac(odd * k, 2 * (int64_t)n);
        }
}

/* Per-coefficient factor applied to G_n in the requested direction/norm.
 * forward ORTHO: alpha_k (Eq. 1);  forward NONE: 2;
 * inverse ORTHO: alpha_k;          inverse NONE: 1 for k = 0, else 2. */
static double coef_scale(int n, int k, int dir, int norm)
{
    if (norm == ORACLE_NORM_ORTHO) {
        if (k == 0 && g_fault != 1) return sqrt(1.0 / n);
        return sqrt(2.0 / n);
    }
    if (dir == ORACLE_DIR_FORWARD) return 2.0;
    return (k == 0) ? 1.0 : 2.0;
}

/* The 1D operator matrix M (n x n, row-major) so that the 2D result is
 * M_h X M_w^T:
 *   forward: M[k][j] = s_k G[k][j]      (ORTHO: M = Q_n)
 *   inverse: M[j][k] = s_k G[k][j]      (ORTHO: M = Q_n^T)                 */
void oracle_matrix(int n, int dir, int norm, double *M)
{
    double *G = (double *)malloc(sizeof(double) * (size_t)n * n);
    basis(n, G);
    for (int k = 0; k < n; ++k) {
        double s = coef_scale(n, k, dir, norm);
        for (int j = 0; j < n; ++j) {
            double v = s * G[(size_t)k * n + j];
            int transpose = (dir == ORACLE_DIR_INVERSE) && (g_fault != 4);
            if (transpose) M[(size_t)j * n + k] = v;
            else M[(size_t)k * n + j] = v;
        }
    }
    free(G);
}

/* The two passes of Eq. 2 for one array, out = Mh X Mw^T, split into row
 * ranges so that one array can be shared by several threads.  Every output
 * element is one plain double sum in index order (j in pass 1, i in pass 2),
 * whatever the split; the intermediate T is kept transposed (Tt[l][i]) only so
 * that pass 2 reads it contiguously.
 *
 * Pass 1, rows i0 .. i1-1:  T[i][l] = sum_j X[i][j] Mw[l][j]  (stored Tt[l][i]).
 * The input is float (xf) or double (xd, the round trip's second half).      */
static void pass_rows(int h, int w, const double *Mw, const float *xf, const double *xd,
                      double *Tt, int i0, int i1)
{
    int last_w = (g_fault == 2) ? w - 1 : w;
    for (int i = i0; i < i1; ++i) {
        const float *rf = xf ? xf + (size_t)i * w : NULL;
        const double *rd = xd ? xd + (size_t)i * w : NULL;
        int l = 0;
        /* four outputs at a time: four independent sums, each in j order */
        for (; l + 4 <= w; l += 4) {
            const double *m0 = Mw + (size_t)l * w, *m1 = m0 + w, *m2 = m1 + w, *m3 = m2 + w;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            for (int j = 0; j < last_w; ++j) {
                double x = rf ? (double)rf[j] : rd[j];
                a0 += x * m0[j];
                a1 += x * m1[j];
                a2 += x * m2[j];
                a3 += x * m3[j];
            }
            Tt[(size_t)l * h + i] = a0;
            Tt[(size_t)(l + 1) * h + i] = a1;
            Tt[(size_t)(l + 2) * h + i] = a2;
            Tt[(size_t)(l + 3) * h + i] = a3;
        }
        for (; l < w; ++l) {
            const double *m0 = Mw + (size_t)l * w;
            double a0 = 0.0;
            for (int j = 0; j < last_w; ++j) a0 += (rf ? (double)rf[j] : rd[j]) * m0[j];
            Tt[(size_t)l * h + i] = a0;
        }
    }
}

/* Pass 2, output rows k0 .. k1-1:  out[k][l] = sum_i Mh[k][i] T[i][l]. */
static void pass_cols(int h, int w, const double *Mh, const double *Tt, double *out, int k0, int k1)
{
    int last_h = (g_fault == 2) ? h - 1 : h;
    for (int k = k0; k < k1; ++k) {
        const double *mk = Mh + (size_t)k * h;
        int l = 0;
        for (; l + 4 <= w; l += 4) {
            const double *t0 = Tt + (size_t)l * h, *t1 = t0 + h, *t2 = t1 + h, *t3 = t2 + h;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            for (int i = 0; i < last_h; ++i) {
                double m = mk[i];
                a0 += m * t0[i];
                a1 += m * t1[i];
                a2 += m * t2[i];
                a3 += m * t3[i];
            }
            out[(size_t)k * w + l] = a0;
            out[(size_t)k * w + l + 1] = a1;
            out[(size_t)k * w + l + 2] = a2;
            out[(size_t)k * w + l + 3] = a3;
        }
        for (; l < w; ++l) {
            const double *t0 = Tt + (size_t)l * h;
            double a0 = 0.0;
            for (int i = 0; i < last_h; ++i) a0 += mk[i] * t0[i];
            out[(size_t)k * w + l] = a0;
        }
    }
}

/* The spectral operator of Prop. 1 (Eq. 4): every coefficient Y[k][l] of
 * rows k0 .. k1-1 multiplied by Lambda[k][l] (row-major h x w). */
static void apply_lambda(int h, int w, const double *lam, double *F, int k0, int k1)
{
    for (int k = k0; k < k1; ++k)
        for (int l = 0; l < w; ++l) {
            size_t at = (g_fault == 6) ? (size_t)l * h + k : (size_t)k * w + l;
            F[(size_t)k * w + l] *= lam[at];
        }
}

/* Work shared by the threads of one call.  Arrays are dealt out whole to
 * threads when there are at least as many arrays as threads; otherwise the
 * threads share each array, splitting both passes by rows (a barrier between
 * the passes). */
typedef struct {
    int h, w, nthreads;
    const double *Mh, *Mw, *Mh2, *Mw2;
    const float *in;
    double *out;
    int64_t batch;
    int roundtrip;
    const double *lam;       /* round trip with a spectral diagonal (Eq. 4), or NULL */
    int shared;              /* 1: threads share each array */
    double *Tt, *F;          /* shared mode: the intermediates of the current array */
    pthread_barrier_t bar;
} call_t;

typedef struct {
    call_t *c;
    int t;
} job_t;

static void range_of(int n, int parts, int t, int *a, int *b)
{
    int per = n / parts, rem = n % parts;
    *a = t * per + (t < rem ? t : rem);
    *b = *a + per + (t < rem ? 1 : 0);
}

static void *worker(void *arg)
{
    job_t *jb = (job_t *)arg;
    call_t *c = jb->c;
    const int h = c->h, w = c->w;
    const size_t hw = (size_t)h * w;
    if (!c->shared) {
        double *Tt = (double *)malloc(sizeof(double) * hw);
        double *F = c->roundtrip ? (double *)malloc(sizeof(double) * hw) : NULL;
        int64_t per = c->batch / c->nthreads, rem = c->batch % c->nthreads;
        int64_t first = jb->t * per + (jb->t < rem ? jb->t : rem);
        int64_t last = first + per + (jb->t < rem ? 1 : 0);
        for (int64_t b = first; b < last; ++b) {
            const float *x = c->in + (size_t)b * hw;
            double *y = c->out + (size_t)b * hw;
            if (!c->roundtrip) {
                pass_rows(h, w, c->Mw, x, NULL, Tt, 0, h);
                pass_cols(h, w, c->Mh, Tt, y, 0, h);
            } else {
                pass_rows(h, w, c->Mw, x, NULL, Tt, 0, h);
                pass_cols(h, w, c->Mh, Tt, F, 0, h);
                if (c->lam) apply_lambda(h, w, c->lam, F, 0, h);
                pass_rows(h, w, c->Mw2, NULL, F, Tt, 0, h);
                pass_cols(h, w, c->Mh2, Tt, y, 0, h);
            }
        }
        free(Tt);
        free(F);
        return NULL;
    }
    int r0, r1;
    range_of(h, c->nthreads, jb->t, &r0, &r1);
    for (int64_t b = 0; b < c->batch; ++b) {
        const float *x = c->in + (size_t)b * hw;
        double *y = c->out + (size_t)b * hw;
        pass_rows(h, w, c->Mw, x, NULL, c->Tt, r0, r1);
        pthread_barrier_wait(&c->bar);
        if (!c->roundtrip) {
            pass_cols(h, w, c->Mh, c->Tt, y, r0, r1);
        } else {
            pass_cols(h, w, c->Mh, c->Tt, c->F, r0, r1);
            if (c->lam) apply_lambda(h, w, c->lam, c->F, r0, r1);
            pthread_barrier_wait(&c->bar);
            pass_rows(h, w, c->Mw2, NULL, c->F, c->Tt, r0, r1);
            pthread_barrier_wait(&c->bar);
            pass_cols(h, w, c->Mh2, c->Tt, y, r0, r1);
        }
        pthread_barrier_wait(&c->bar); /* Tt is reused by the next array */
    }
    return NULL;
}

int oracle_default_threads(void)
{
    cpu_set_t set;
    if (sched_getaffinity(0, sizeof(set), &set) == 0) {
        int c = CPU_COUNT(&set);
        if (c > 0) return c;
    }
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static int run_jobs(int h, int w, int dir, int norm, const float *in, double *out,
                    int64_t batch, int threads, int roundtrip, const double *lam)
{
    if (h < 1 || w < 1 || batch < 0) return -1;
    if (batch == 0) return 0;
    if (threads <= 0) threads = oracle_default_threads();
    if (threads > 512) threads = 512;
    int shared = 0;
    if (threads > batch) {
        /* fewer arrays than threads: share each array when it is big enough
         * to be worth it, else use one thread per array */
        if ((int64_t)h * w >= 65536 && h >= 2) {
            shared = 1;
            if (threads > h) threads = h;
        } else {
            threads = (int)batch;
        }
    }

    double *Mh = (double *)malloc(sizeof(double) * (size_t)h * h);
    double *Mw = (double *)malloc(sizeof(double) * (size_t)w * w);
    double *Mh2 = NULL, *Mw2 = NULL;
    int d1 = roundtrip ? ORACLE_DIR_FORWARD : dir;
    oracle_matrix(h, d1, norm, Mh);
    oracle_matrix(w, d1, norm, Mw);
    if (g_fault == 5 && h != w) { /* planted fault: row axis uses the column matrix */
        free(Mw);
        Mw = (double *)malloc(sizeof(double) * (size_t)w * w);
        for (int a = 0; a < w; ++a)
            for (int b = 0; b < w; ++b)
                Mw[(size_t)a * w + b] = (a < h && b < h) ? Mh[(size_t)a * h + b] : 0.0;
    }
    if (roundtrip) {
        Mh2 = (double *)malloc(sizeof(double) * (size_t)h * h);
        Mw2 = (double *)malloc(sizeof(double) * (size_t)w * w);
        oracle_matrix(h, ORACLE_DIR_INVERSE, norm, Mh2);
        oracle_matrix(w, ORACLE_DIR_INVERSE, norm, Mw2);
        if (norm == ORACLE_NORM_NONE) { /* normalized round trip: divide by 4hw */
            double s = 1.0 / (4.0 * (double)h * (double)w);
            for (size_t q = 0; q < (size_t)h * h; ++q) Mh2[q] *= s;
        }
    }

    call_t c;
    memset(&c, 0, sizeof(c));
    c.h = h; c.w = w; c.nthreads = threads;
    c.Mh = Mh; c.Mw = Mw; c.Mh2 = Mh2; c.Mw2 = Mw2;
    c.in = in; c.out = out; c.batch = batch; c.roundtrip = roundtrip; c.shared = shared;
    c.lam = lam;
    if (shared) {
        c.Tt = (double *)malloc(sizeof(double) * (size_t)h * w);
        c.F = roundtrip ? (double *)malloc(sizeof(double) * (size_t)h * w) : NULL;
        pthread_barrier_init(&c.bar, NULL, (unsigned)threads);
    }
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * threads);
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * threads);
    for (int t = 0; t < threads; ++t) { jobs[t].c = &c; jobs[t].t = t; }
    for (int t = 1; t < threads; ++t) pthread_create(&tid[t], NULL, worker, &jobs[t]);
    worker(&jobs[0]);
    for (int t = 1; t < threads; ++t) pthread_join(tid[t], NULL);
    if (shared) {
        pthread_barrier_destroy(&c.bar);
        free(c.Tt);
        free(c.F);
    }
    free(tid);
    free(jobs);
    free(Mh);
    free(Mw);
    free(Mh2);
    free(Mw2);
    return 0;
}

/* Forward 2D DCT-II of `batch` contiguous h x w float arrays into double. */
int oracle_forward(int h, int w, int norm, const float *in, double *out, int64_t batch, int threads)
{
    return run_jobs(h, w, ORACLE_DIR_FORWARD, norm, in, out, batch, threads, 0, NULL);
}

/* Inverse 2D DCT-III of `batch` contiguous h x w float arrays into double. */
int oracle_inverse(int h, int w, int norm, const float *in, double *out, int64_t batch, int threads)
{
    return run_jobs(h, w, ORACLE_DIR_INVERSE, norm, in, out, batch, threads, 0, NULL);
}

/* FP64 composition C^{-1}(C(X)) (normalized); its exact result is X. */
int oracle_roundtrip(int h, int w, int norm, const float *in, double *out, int64_t batch, int threads)
{
    return run_jobs(h, w, ORACLE_DIR_FORWARD, norm, in, out, batch, threads, 1, NULL);
}

/* Transform -- spectral operator -- inverse (Prop. 1, Eq. 4):
 * out = U^T Lambda U X = Q_h^T (Lambda o (Q_h X Q_w^T)) Q_w for every array,
 * with the orthonormal Q of Eq. 1 and `lam` the h x w diagonal (row-major,
 * Lambda[k][l] multiplies coefficient (k, l)).  Lambda = 1 gives the round
 * trip, whose exact result is X. */
int oracle_spectral(int h, int w, const double *lam, const float *in, double *out, int64_t batch, int threads)
{
    if (!lam) return -1;
    return run_jobs(h, w, ORACLE_DIR_FORWARD, ORACLE_NORM_ORTHO, in, out, batch, threads, 1, lam);
}

/* Brute-force O(h^2 w^2) double sum of Eq. 2 for one array, with every cosine
 * taken directly from libm (no table, no separable factoring). */
int oracle_bruteforce(int h, int w, int dir, int norm, const float *in, double *out)
{
    if (h < 1 || w < 1) return -1;
    for (int p = 0; p < h; ++p)
        for (int q = 0; q < w; ++q) {
            double acc = 0.0;
            for (int a = 0; a < h; ++a)
                for (int b = 0; b < w; ++b) {
                    /* forward: out[k=p][l=q] += s_k s_l x[i=a][j=b] cos(..a..p) cos(..b..q)
                     * inverse: out[i=p][j=q] += s_k s_l y[k=a][l=b] cos(..p..a) cos(..q..b) */
                    int k, i, l, j;
                    if (dir == ORACLE_DIR_FORWARD) { k = p; i = a; l = q; j = b; }
                    else { k = a; i = p; l = b; j = q; }
                    double sk, sl;
                    if (norm == ORACLE_NORM_ORTHO) {
                        sk = (k == 0) ? 1.0 / sqrt((double)h) : sqrt(2.0 / h);
                        sl = (l == 0) ? 1.0 / sqrt((double)w) : sqrt(2.0 / w);
                    } else if (dir == ORACLE_DIR_FORWARD) {
                        sk = 2.0; sl = 2.0;
                    } else {
                        sk = (k == 0) ? 1.0 : 2.0;
                        sl = (l == 0) ? 1.0 : 2.0;
                    }
                    double ch = cos(M_PI * (2.0 * i + 1.0) * k / (2.0 * h));
                    double cw = cos(M_PI * (2.0 * j + 1.0) * l / (2.0 * w));
                    acc += sk * sl * (double)in[(size_t)a * w + b] * ch * cw;
                }
            out[(size_t)p * w + q] = acc;
        }
    return 0;
}
