/*
 * Direct O(L^2) FP64 linear convolution in plain C: the definition of the
 * result of a hybrid-dealiased convolution (Section 2: (f*g)_j = sum_i f_i
 * g_{j-i}; Section 3 centered; Section 4 Hermitian), written out.
 *
 * TEST INFRASTRUCTURE ONLY.  This is part of the CPU oracle.  It shares no
 * code with the CUDA library and is never linked into it; the tests, the
 * smoke check and the benchmark's CPU-baseline leg load it through ctypes.
 *
 * Layout: complex numbers are interleaved (re, im) doubles.  Each input a has
 * `count` instances of `n` stored values, instance b starting at
 * f[a] + 2*b*n.  Stored values are:
 *   kind 0 (complex):   f_0 .. f_{L-1},               n = L
 *   kind 1 (centered):  f_c at stored j = c + L/2,     n = L
 *   kind 2 (Hermitian): f_0 .. f_{H-1}, f_{-c} = conj f_c, Im f_0 ignored,
 *                       n = H = ceil(L/2)
 * mult 0: h = f1*f2 (A = 2); mult 1: h = f1*f2 + f2*f3 + f3*f1 (A = 3).
 * The output h has the stored layout of the inputs.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double re, im;
} cplx;

/* value of a stored array at "full" index k of the linear layout the
 * convolution is taken in (complex/centered: the stored array itself;
 * Hermitian: the expanded array of length 2H-1, centered at H-1) */
static cplx at(const double* f, int kind, int64_t n, int64_t k) {
    cplx z = {0.0, 0.0};
    if (kind != 2) {
        if (k >= 0 && k < n) {
            z.re = f[2 * k];
            z.im = f[2 * k + 1];
        }
        return z;
    }
    int64_t c = k - (n - 1);
    if (c >= 0 && c < n) {
        z.re = f[2 * c];
        z.im = (c == 0) ? 0.0 : f[2 * c + 1];
    } else if (c < 0 && -c < n) {
        z.re = f[2 * (-c)];
        z.im = -f[2 * (-c) + 1];
    }
    return z;
}

/* one output value: sum_i a(i) b(k - i) over the linear layout of length Le */
static cplx pair_sum(const double* a, const double* b, int kind, int64_t n, int64_t Le, int64_t k) {
    int64_t lo = k - (Le - 1);
    if (lo < 0) lo = 0;
    int64_t hi = k < Le - 1 ? k : Le - 1;
    double sr = 0.0, si = 0.0;
    for (int64_t i = lo; i <= hi; ++i) {
        cplx x = at(a, kind, n, i);
        cplx y = at(b, kind, n, k - i);
        sr += x.re * y.re - x.im * y.im;
        si += x.re * y.im + x.im * y.re;
    }
    cplx z = {sr, si};
    return z;
}

static void conv_one(int kind, int mult, int64_t L, int64_t n, const double* const* f, double* h) {
    int64_t Le = (kind == 2) ? 2 * n - 1 : n;      /* linear layout length */
    int64_t off;                                    /* full index of stored output 0 */
    if (kind == 0) off = 0;
    else if (kind == 1) off = L / 2;
    else off = 2 * (n - 1);
    for (int64_t j = 0; j < n; ++j) {
        int64_t k = j + off;
        cplx s = pair_sum(f[0], f[1], kind, n, Le, k);
        if (mult == 1) {
            cplx s2 = pair_sum(f[1], f[2], kind, n, Le, k);
            cplx s3 = pair_sum(f[2], f[0], kind, n, Le, k);
            s.re += s2.re + s3.re;
            s.im += s2.im + s3.im;
        }
        h[2 * j] = s.re;
        h[2 * j + 1] = s.im;
    }
}

typedef struct {
    int kind, mult, A;
    int64_t L, n, count;
    const double* const* f;
    double* h;
    int64_t begin, end;
} job;

static void* worker(void* arg) {
    job* jb = (job*)arg;
    const double* ptrs[3];
    for (int64_t b = jb->begin; b < jb->end; ++b) {
        for (int a = 0; a < jb->A; ++a) ptrs[a] = jb->f[a] + 2 * b * jb->n;
        conv_one(jb->kind, jb->mult, jb->L, jb->n, ptrs, jb->h + 2 * b * jb->n);
    }
    return NULL;
}

/* Returns 0 on success, -1 on bad arguments. */
int oracle_conv1d_batch(int kind, int mult, int64_t L, int64_t count, const double* const* f, double* h,
                        int nthreads) {
    if (kind < 0 || kind > 2 || mult < 0 || mult > 1 || L <= 0 || count < 0) return -1;
    int A = mult == 0 ? 2 : 3;
    int64_t n = (kind == 2) ? (L + 1) / 2 : L;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (count < nthreads) nthreads = (int)(count > 0 ? count : 1);
    pthread_t th[256];
    job jobs[256];
    int64_t per = (count + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].kind = kind;
        jobs[t].mult = mult;
        jobs[t].A = A;
        jobs[t].L = L;
        jobs[t].n = n;
        jobs[t].count = count;
        jobs[t].f = f;
        jobs[t].h = h;
        jobs[t].begin = t * per < count ? t * per : count;
        jobs[t].end = (t + 1) * per < count ? (t + 1) * per : count;
        pthread_create(&th[t], NULL, worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* Selected stored output indices of instance 0 (O(L) per point). */
int oracle_conv1d_points(int kind, int mult, int64_t L, const double* const* f, const int64_t* idx, int64_t npts,
                         double* out) {
    if (kind < 0 || kind > 2 || mult < 0 || mult > 1 || L <= 0) return -1;
    int64_t n = (kind == 2) ? (L + 1) / 2 : L;
    int64_t Le = (kind == 2) ? 2 * n - 1 : n;
    int64_t off = (kind == 0) ? 0 : (kind == 1 ? L / 2 : 2 * (n - 1));
    for (int64_t p = 0; p < npts; ++p) {
        if (idx[p] < 0 || idx[p] >= n) return -1;
        int64_t k = idx[p] + off;
        cplx s = pair_sum(f[0], f[1], kind, n, Le, k);
        if (mult == 1) {
            cplx s2 = pair_sum(f[1], f[2], kind, n, Le, k);
            cplx s3 = pair_sum(f[2], f[0], kind, n, Le, k);
            s.re += s2.re + s3.re;
            s.im += s2.im + s3.im;
        }
        out[2 * p] = s.re;
        out[2 * p + 1] = s.im;
    }
    return 0;
}
