/*
 * timing_mt.c -- the oracle's red-black SOR sweep (Eq. 7 in red-black order) with its row
 * loop split across host threads: a timing wrapper for the all-cores CPU baseline.
 *
 * TEST INFRASTRUCTURE, like oracle.c: only the test suite and the benchmark's CPU-baseline
 * leg may load it. oracle.c stays single-threaded and plain; this file repeats its
 * red-black SOR update expression (the same operations and roundings:
 * s = fma(b2, N + S, E + W); psi = fma(w, s * (1/d), (1 - w) * psi)) so that the threaded
 * sweeps are bitwise the oracle's (a CPU test checks this), and adds only the threading:
 * each thread owns a contiguous band of rows, and a barrier separates the red pass from
 * the black pass (within one colour no point reads another point of its colour).
 * Build with -ffp-contract=off, like oracle.c.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>

#define AT(a, m, i, j) ((a)[(size_t)(j) * (size_t)(m) + (size_t)(i)])

typedef struct {
    int m, n, j0, j1, nsweeps;
    double b2, inv_d, w, one_minus_w;
    double* psi;
    pthread_barrier_t* barrier;
} band_t;

static void colour_pass(const band_t* b, int colour)
{
    const int m = b->m;
    double* psi = b->psi;
    for (int j = b->j0; j < b->j1; ++j)
        for (int i = 1 + ((1 + j + colour) & 1); i < m - 1; i += 2) {
            double ew = AT(psi, m, i - 1, j) + AT(psi, m, i + 1, j);
            double ns = AT(psi, m, i, j - 1) + AT(psi, m, i, j + 1);
            double s = fma(b->b2, ns, ew);
            double gs = s * b->inv_d;
            AT(psi, m, i, j) = fma(b->w, gs, b->one_minus_w * AT(psi, m, i, j));
        }
}

static void* band_main(void* arg)
{
    const band_t* b = (const band_t*)arg;
    for (int k = 0; k < b->nsweeps; ++k)
        for (int c = 0; c < 2; ++c) {
            colour_pass(b, c);
            pthread_barrier_wait(b->barrier);
        }
    return NULL;
}

/* nsweeps red-black SOR sweeps of psi (m x n, row-major, ring fixed) on nthreads threads.
 * Returns 0, or -1 if the threads cannot be started. */
int ora_mt_sor_rb_sweeps(int m, int n, double beta, double w, int nsweeps, double* psi,
                         int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n - 2) nthreads = n - 2 > 0 ? n - 2 : 1;
    const double b2 = beta * beta, d = 2.0 * (1.0 + b2);
    pthread_barrier_t barrier;
    if (pthread_barrier_init(&barrier, NULL, (unsigned)nthreads) != 0) return -1;
    band_t* bands = (band_t*)calloc((size_t)nthreads, sizeof(band_t));
    pthread_t* tids = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!bands || !tids) {
        free(bands);
        free(tids);
        pthread_barrier_destroy(&barrier);
        return -1;
    }
    const int rows = n - 2;
    for (int t = 0; t < nthreads; ++t) {
        band_t* b = &bands[t];
        b->m = m;
        b->n = n;
        b->j0 = 1 + (int)((long long)rows * t / nthreads);
        b->j1 = 1 + (int)((long long)rows * (t + 1) / nthreads);
        b->nsweeps = nsweeps;
        b->b2 = b2;
        b->inv_d = 1.0 / d;
        b->w = w;
        b->one_minus_w = 1.0 - w;
        b->psi = psi;
        b->barrier = &barrier;
    }
    int started = 0, rc = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&tids[t], NULL, band_main, &bands[t]) != 0) {
            rc = -1;
            break;
        }
        ++started;
    }
    if (rc == 0) {
        band_main(&bands[0]);
    }
    for (int t = 1; t <= started; ++t) pthread_join(tids[t], NULL);
    free(bands);
    free(tids);
    pthread_barrier_destroy(&barrier);
    return rc;
}
