/*
 * p3_oracle.c -- plain, slow, FP64 CPU oracle for the 3D real-to-complex
 * forward transform and its complex-to-real inverse described in the P3DFFT
 * paper (Pekurovsky, "P3DFFT: a framework for parallel computations of Fourier
 * transforms in three dimensions").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (Sect. 2, Sect. 3.2, Table 1):
 *   forward:  F[kz][ky][kx] = sum_{x,y,z} f[z][y][x]
 *                  * exp(-2 pi i (kx x/Nx + ky y/Ny + kz z/Nz)),
 *             kx in [0, H), H = floor(Nx/2)+1 (the paper's (Nx+2)/2 with
 *             integer division, Sect. 3.2), done as three passes of 1D
 *             transforms in X, then Y, then Z (Sect. 2, Fig. 2).
 *   Z may instead be the Chebyshev transform (Sect. 2 last paragraph,
 *             Sect. 3.1), taken as the unnormalised DCT-I on Gauss-Lobatto
 *             points:  Y_n = x_0 + (-1)^n x_M + 2 sum_{j=1}^{M-1} x_j cos(pi j n/M),
 *             M = Nz-1, applied to real and imaginary parts alike, evaluated
 *             as the direct O(M^2) sum.
 *   Z may instead be the sine transform (the "sine" of Sect. 3.1's
 *             sine/cosine transforms), taken as the unnormalised DST-I of the
 *             Nz interior points of a Dirichlet grid:
 *             Y_k = 2 sum_{j=0}^{Nz-1} x_j sin(pi (j+1)(k+1)/(Nz+1)),
 *             again as the direct O(Nz^2) sum.
 *   Y or Z may be the "empty" (identity) transform (Sect. 3.1).
 *   backward: the reverse order (Z, Y inverse with the + sign, then X c2r),
 *             where the X c2r of a line is f[x] = Re sum_{k<H} w_k F[k]
 *             exp(+2 pi i k x/Nx), w_0 = 1, w_{Nx/2} = 1 for even Nx and
 *             w_k = 2 otherwise.  Both directions are unnormalised, so a round
 *             trip returns the input times a scale factor (Sect. 4.1).
 *
 * The 1D FFT is textbook recursive decimation in time (Cooley-Tukey): split
 * n = p*m with p the smallest prime factor of n, transform the p decimated
 * subsequences, and recombine each output as a p-term sum.  A prime length is
 * therefore a naive O(n^2) DFT.  Roots of unity come from cosl/sinl of the
 * exactly reduced angle 2 pi (t mod n)/n.
 *
 * All arrays are C row-major with the rightmost index fastest:
 *   real  [Nz][Ny][Nx],  complex (XYZ storage)  [Nz][Ny][H].
 *
 * Parity: pinned by tests/test_oracle_pins.py against brute-force O(N^2)
 * sums, closed-form plane-wave and Chebyshev-polynomial deltas, Parseval,
 * Hermitian symmetry, linearity and the forward-inverse round trip.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { P3O_FFT = 0, P3O_CHEB = 1, P3O_EMPTY = 2, P3O_SINE = 3 };

/* ------------------------------------------------------------------------- */
/* Roots of unity: roots[t] = exp(sign * 2 pi i t / n), t in [0, n).           */
/* ------------------------------------------------------------------------- */
static cplx* make_roots(long n, int sign)
{
    cplx* r = (cplx*)malloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1));
    if (!r) return NULL;
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (long t = 0; t < n; ++t) {
        long double a = two_pi * (long double)t / (long double)n;
        r[t] = (double)cosl(a) + (double)sign * (double)sinl(a) * I;
    }
    return r;
}

static long smallest_prime_factor(long n)
{
    for (long p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/*
 * Decimation-in-time recursion.  x is read with stride xs; X (length n,
 * contiguous) receives the transform.  roots holds W_N^t for the top-level
 * length N; the current length n divides N, so W_n^t = roots[(t mod n) * (N/n)].
 * tmp must hold at least 2n entries.
 */
static void fft_rec(long n, const cplx* x, long xs, cplx* X,
                    const cplx* roots, long N, cplx* tmp)
{
    if (n == 1) {
        X[0] = x[0];
        return;
    }
    long p = smallest_prime_factor(n);
    long m = n / p;
    /* Y_r = DFT_m of the subsequence x[r + p j], j < m, stored at X[r m ...]. */
    for (long r = 0; r < p; ++r)
        fft_rec(m, x + r * xs, xs * p, X + r * m, roots, N, tmp + n);
    memcpy(tmp, X, sizeof(cplx) * (size_t)n);
    long step = N / n;
    for (long q = 0; q < p; ++q) {
        for (long k = 0; k < m; ++k) {
            long kk = k + m * q;
            cplx acc = 0.0;
            for (long r = 0; r < p; ++r) {
                long t = (r * kk) % n;
                acc += roots[t * step] * tmp[r * m + k];
            }
            X[kk] = acc;
        }
    }
}

/* One 1D complex transform of length n: out = DFT(in) with exp(sign 2 pi i..). */
static void fft1d_with(long n, const cplx* in, long is, cplx* out,
                       const cplx* roots, cplx* tmp)
{
    fft_rec(n, in, is, out, roots, n, tmp);
}

/* ------------------------------------------------------------------------- */
/* A minimal fork-join over a line range.                                      */
/* ------------------------------------------------------------------------- */
typedef void (*line_fn)(void* ctx, long l0, long l1);

typedef struct {
    line_fn fn;
    void* ctx;
    long l0, l1;
} job_t;

static void* job_main(void* a)
{
    job_t* j = (job_t*)a;
    j->fn(j->ctx, j->l0, j->l1);
    return NULL;
}

static void parallel_lines(line_fn fn, void* ctx, long l0, long l1, int nthreads)
{
    long n = l1 - l0;
    if (n <= 0) return;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((long)nthreads > n) nthreads = (int)n;
    if (nthreads == 1) {
        fn(ctx, l0, l1);
        return;
    }
    pthread_t th[256];
    job_t jobs[256];
    int started[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].l0 = l0 + n * t / nthreads;
        jobs[t].l1 = l0 + n * (t + 1) / nthreads;
        started[t] = pthread_create(&th[t], NULL, job_main, &jobs[t]) == 0;
        if (!started[t]) fn(ctx, jobs[t].l0, jobs[t].l1);
    }
    for (int t = 0; t < nthreads; ++t)
        if (started[t]) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------- */
/* Line addressing: line L starts at (L / per) * gstride + (L % per) * lstride */
/* and its elements are es apart.                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
    long per, gstride, lstride, es;
} lines_t;

static long line_base(const lines_t* g, long L)
{
    return (L / g->per) * g->gstride + (L % g->per) * g->lstride;
}

/* --- X stage, forward: each real row of Nx -> H complex bins ------------- */
typedef struct {
    long nx, H;
    const double* f;
    cplx* F;
    const cplx* roots;
} xr2c_ctx;

static void xr2c_lines(void* c, long l0, long l1)
{
    xr2c_ctx* k = (xr2c_ctx*)c;
    long nx = k->nx;
    cplx* line = (cplx*)malloc(sizeof(cplx) * (size_t)nx);
    cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)nx);
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)(2 * nx));
    for (long L = l0; L < l1; ++L) {
        const double* row = k->f + L * nx;
        for (long x = 0; x < nx; ++x) line[x] = row[x];
        fft1d_with(nx, line, 1, out, k->roots, tmp);
        memcpy(k->F + L * k->H, out, sizeof(cplx) * (size_t)k->H);
    }
    free(line);
    free(out);
    free(tmp);
}

/* --- X stage, inverse: H complex bins -> real row via the weighted-Re sum -- */
typedef struct {
    long nx, H;
    const cplx* F;
    double* f;
    const cplx* roots; /* + sign */
} xc2r_ctx;

static void xc2r_lines(void* c, long l0, long l1)
{
    xc2r_ctx* k = (xc2r_ctx*)c;
    long nx = k->nx, H = k->H;
    cplx* G = (cplx*)malloc(sizeof(cplx) * (size_t)nx);
    cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)nx);
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)(2 * nx));
    for (long L = l0; L < l1; ++L) {
        const cplx* row = k->F + L * H;
        /* G[k] = w_k F[k] for k < H, zero above: Re of its inverse DFT is the
           weighted-Re sum written in the file header. */
        for (long q = 0; q < nx; ++q) G[q] = 0.0;
        for (long q = 0; q < H; ++q) {
            double w = 2.0;
            if (q == 0) w = 1.0;
            if (nx % 2 == 0 && q == nx / 2) w = 1.0;
            G[q] = w * row[q];
        }
        fft1d_with(nx, G, 1, out, k->roots, tmp);
        double* dst = k->f + L * nx;
        for (long x = 0; x < nx; ++x) dst[x] = creal(out[x]);
    }
    free(G);
    free(out);
    free(tmp);
}

/* --- complex lines: in-place c2c along one axis ------------------------- */
typedef struct {
    long n;
    lines_t g;
    cplx* data;
    const cplx* roots;
} c2c_ctx;

static void c2c_lines(void* c, long l0, long l1)
{
    c2c_ctx* k = (c2c_ctx*)c;
    long n = k->n;
    cplx* line = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)(2 * n));
    for (long L = l0; L < l1; ++L) {
        cplx* p = k->data + line_base(&k->g, L);
        for (long e = 0; e < n; ++e) line[e] = p[e * k->g.es];
        fft1d_with(n, line, 1, out, k->roots, tmp);
        for (long e = 0; e < n; ++e) p[e * k->g.es] = out[e];
    }
    free(line);
    free(out);
    free(tmp);
}

/* --- complex lines: in-place DCT-I (direct sum) along one axis ---------- */
typedef struct {
    long n; /* points per line = M + 1 */
    lines_t g;
    cplx* data;
    const double* cosv; /* cos(pi t / M), t in [0, 2M) */
} dct_ctx;

static void dct1_lines(void* c, long l0, long l1)
{
    dct_ctx* k = (dct_ctx*)c;
    long n = k->n, M = n - 1;
    cplx* line = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    for (long L = l0; L < l1; ++L) {
        cplx* p = k->data + line_base(&k->g, L);
        for (long e = 0; e < n; ++e) line[e] = p[e * k->g.es];
        for (long q = 0; q < n; ++q) {
            cplx acc = line[0] + ((q % 2) ? -line[M] : line[M]);
            for (long j = 1; j < M; ++j) acc += 2.0 * k->cosv[(j * q) % (2 * M)] * line[j];
            p[q * k->g.es] = acc;
        }
    }
    free(line);
}

static double* make_cheb_cos(long M)
{
    double* c = (double*)malloc(sizeof(double) * (size_t)(2 * M));
    if (!c) return NULL;
    const long double pi = 3.141592653589793238462643383279502884L;
    for (long t = 0; t < 2 * M; ++t) c[t] = (double)cosl(pi * (long double)t / (long double)M);
    return c;
}

/* --- complex lines: in-place DST-I (direct sum) along one axis ---------- */
typedef struct {
    long n; /* points per line */
    lines_t g;
    cplx* data;
    const double* sinv; /* sin(pi t / (n+1)), t in [0, 2(n+1)) */
} dst_ctx;

static void dst1_lines(void* c, long l0, long l1)
{
    dst_ctx* k = (dst_ctx*)c;
    long n = k->n, P = 2 * (n + 1);
    cplx* line = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    for (long L = l0; L < l1; ++L) {
        cplx* p = k->data + line_base(&k->g, L);
        for (long e = 0; e < n; ++e) line[e] = p[e * k->g.es];
        for (long q = 0; q < n; ++q) {
            cplx acc = 0;
            for (long j = 0; j < n; ++j) acc += 2.0 * k->sinv[((j + 1) * (q + 1)) % P] * line[j];
            p[q * k->g.es] = acc;
        }
    }
    free(line);
}

static double* make_sine(long n)
{
    long P = 2 * (n + 1);
    double* v = (double*)malloc(sizeof(double) * (size_t)P);
    if (!v) return NULL;
    const long double pi = 3.141592653589793238462643383279502884L;
    for (long t = 0; t < P; ++t) v[t] = (double)sinl(pi * (long double)t / (long double)(n + 1));
    return v;
}

/* ------------------------------------------------------------------------- */
/* Public entry points (plain C ABI, called through ctypes by the tests).      */
/* Return 0 on success, -1 on bad arguments, -2 on allocation failure.         */
/* ------------------------------------------------------------------------- */

/* 1D complex DFT, out[k] = sum_j in[j] exp(sign 2 pi i j k / n). */
int p3o_fft1d(long n, const cplx* in, cplx* out, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1)) return -1;
    cplx* roots = make_roots(n, sign);
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)(2 * n));
    if (!roots || !tmp) { free(roots); free(tmp); return -2; }
    fft1d_with(n, in, 1, out, roots, tmp);
    free(roots);
    free(tmp);
    return 0;
}

/* 1D unnormalised DCT-I of n = M+1 complex points (direct sum). */
int p3o_dct1(long n, const cplx* in, cplx* out)
{
    if (n < 2) return -1;
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    double* cosv = make_cheb_cos(n - 1);
    if (!buf || !cosv) { free(buf); free(cosv); return -2; }
    memcpy(buf, in, sizeof(cplx) * (size_t)n);
    dct_ctx k = { n, { 1, 0, 0, 1 }, buf, cosv };
    dct1_lines(&k, 0, 1);
    memcpy(out, buf, sizeof(cplx) * (size_t)n);
    free(buf);
    free(cosv);
    return 0;
}

/* 1D unnormalised DST-I of n complex points (direct sum). */
int p3o_dst1(long n, const cplx* in, cplx* out)
{
    if (n < 1) return -1;
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    double* sinv = make_sine(n);
    if (!buf || !sinv) { free(buf); free(sinv); return -2; }
    memcpy(buf, in, sizeof(cplx) * (size_t)n);
    dst_ctx k = { n, { 1, 0, 0, 1 }, buf, sinv };
    dst1_lines(&k, 0, 1);
    memcpy(out, buf, sizeof(cplx) * (size_t)n);
    free(buf);
    free(sinv);
    return 0;
}

/* Forward X stage for rows [r0, r1): f [rows][nx] real -> F [rows][H]. */
int p3o_x_r2c_rows(long nx, const double* f, cplx* F, long r0, long r1, int nthreads)
{
    if (nx < 1 || r0 < 0 || r1 < r0) return -1;
    cplx* roots = make_roots(nx, -1);
    if (!roots) return -2;
    xr2c_ctx k = { nx, nx / 2 + 1, f, F, roots };
    parallel_lines(xr2c_lines, &k, r0, r1, nthreads);
    free(roots);
    return 0;
}

/* Inverse X stage for rows [r0, r1): F [rows][H] -> f [rows][nx] real. */
int p3o_x_c2r_rows(long nx, const cplx* F, double* f, long r0, long r1, int nthreads)
{
    if (nx < 1 || r0 < 0 || r1 < r0) return -1;
    cplx* roots = make_roots(nx, +1);
    if (!roots) return -2;
    xc2r_ctx k = { nx, nx / 2 + 1, F, f, roots };
    parallel_lines(xc2r_lines, &k, r0, r1, nthreads);
    free(roots);
    return 0;
}

/* In-place c2c of lines [l0, l1) of length n; line L starts at
   (L/per)*gstride + (L%per)*lstride, elements es apart. */
int p3o_c2c_lines(long n, long per, long gstride, long lstride, long es,
                  cplx* data, long l0, long l1, int sign, int nthreads)
{
    if (n < 1 || per < 1 || l0 < 0 || l1 < l0 || (sign != 1 && sign != -1)) return -1;
    cplx* roots = make_roots(n, sign);
    if (!roots) return -2;
    c2c_ctx k = { n, { per, gstride, lstride, es }, data, roots };
    parallel_lines(c2c_lines, &k, l0, l1, nthreads);
    free(roots);
    return 0;
}

/* In-place DCT-I of lines [l0, l1) of n = M+1 points; addressing as above. */
int p3o_dct1_lines(long n, long per, long gstride, long lstride, long es,
                   cplx* data, long l0, long l1, int nthreads)
{
    if (n < 2 || per < 1 || l0 < 0 || l1 < l0) return -1;
    double* cosv = make_cheb_cos(n - 1);
    if (!cosv) return -2;
    dct_ctx k = { n, { per, gstride, lstride, es }, data, cosv };
    parallel_lines(dct1_lines, &k, l0, l1, nthreads);
    free(cosv);
    return 0;
}

/* In-place DST-I of lines [l0, l1) of n points; addressing as above. */
int p3o_dst1_lines(long n, long per, long gstride, long lstride, long es,
                   cplx* data, long l0, long l1, int nthreads)
{
    if (n < 1 || per < 1 || l0 < 0 || l1 < l0) return -1;
    double* sinv = make_sine(n);
    if (!sinv) return -2;
    dst_ctx k = { n, { per, gstride, lstride, es }, data, sinv };
    parallel_lines(dst1_lines, &k, l0, l1, nthreads);
    free(sinv);
    return 0;
}

/* Third-dimension / second-dimension pass over a whole XYZ complex array. */
static int yz_pass(long nx, long ny, long nz, int axis, int ttype, int sign,
                   cplx* F, int nthreads)
{
    long H = nx / 2 + 1;
    if (ttype == P3O_EMPTY) return 0;
    if (axis == 1) { /* Y: lines (x, z), base z*ny*H + x, stride H */
        if (ttype != P3O_FFT) return -1;
        return p3o_c2c_lines(ny, H, ny * H, 1, H, F, 0, H * nz, sign, nthreads);
    }
    /* Z: lines (x, y), base y*H + x, stride ny*H */
    if (ttype == P3O_FFT)
        return p3o_c2c_lines(nz, H * ny, 0, 1, ny * H, F, 0, H * ny, sign, nthreads);
    if (ttype == P3O_CHEB)
        return p3o_dct1_lines(nz, H * ny, 0, 1, ny * H, F, 0, H * ny, nthreads);
    if (ttype == P3O_SINE)
        return p3o_dst1_lines(nz, H * ny, 0, 1, ny * H, F, 0, H * ny, nthreads);
    return -1;
}

/* Full forward 3D transform: f [nz][ny][nx] real -> F [nz][ny][H] complex. */
int p3o_forward(long nx, long ny, long nz, int ty, int tz,
                const double* f, cplx* F, int nthreads)
{
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    if (ty != P3O_FFT && ty != P3O_EMPTY) return -1;
    if (tz != P3O_FFT && tz != P3O_CHEB && tz != P3O_EMPTY && tz != P3O_SINE) return -1;
    if (tz == P3O_CHEB && nz < 2) return -1;
    int rc = p3o_x_r2c_rows(nx, f, F, 0, ny * nz, nthreads);
    if (rc) return rc;
    rc = yz_pass(nx, ny, nz, 1, ty, -1, F, nthreads);
    if (rc) return rc;
    return yz_pass(nx, ny, nz, 2, tz, -1, F, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Sampled outputs of the definition for full-size grids.                      */
/* ------------------------------------------------------------------------- */
typedef struct {
    long nx, ny, z0, z1;
    const void* a;  /* chunk [z1-z0][ny][nx] of the given type */
    int type;       /* 0 f32 real, 1 f64 real, 2 complex64, 3 complex128 */
    const cplx* py; /* [ny] phases along y for one index pair */
    const cplx* pz; /* [nz] phases along z (absolute z) */
    cplx* g;        /* [nx] accumulator */
} psum_ctx;

static cplx load_at(const psum_ctx* c, size_t i)
{
    switch (c->type) {
    case 0: return ((const float*)c->a)[i];
    case 1: return ((const double*)c->a)[i];
    case 2: { const float* p = (const float*)c->a + 2 * i; return p[0] + p[1] * I; }
    default: return ((const cplx*)c->a)[i];
    }
}

/* Each worker owns the x range [x0, x1) of the accumulator. */
static void psum_lines(void* v, long x0, long x1)
{
    psum_ctx* c = (psum_ctx*)v;
    for (long z = c->z0; z < c->z1; ++z)
        for (long y = 0; y < c->ny; ++y) {
            const size_t row = ((size_t)(z - c->z0) * (size_t)c->ny + (size_t)y) * (size_t)c->nx;
            const cplx w = c->py[y] * c->pz[z];
            for (long x = x0; x < x1; ++x) c->g[x] += w * load_at(c, row + (size_t)x);
        }
}

/*
 * Accumulate, for nk index pairs (a_k, b_k),
 *   g[k][x] += sum_{z in [z0, z1)} sum_y A[z][y][x] exp(sign 2 pi i (a_k y/ny + b_k z/nz))
 * over a z-chunk A (the rows [z0, z1) of an [nz][ny][nx] array).  With
 * sign -1 and (a, b) = (ky, kz) this is the Y and Z part of the forward
 * definition for one output line; with sign +1, a complex input and
 * (a, b) = (y, z) it is the Y and Z part of the inverse for one real row.
 */
int p3o_phase_sum_yz(long nx, long ny, long nz, const void* chunk, int type, long z0, long z1,
                     long nk, const long* a, const long* b, int sign, cplx* g, int nthreads)
{
    if (nx < 1 || ny < 1 || nz < 1 || z0 < 0 || z1 < z0 || z1 > nz || nk < 1 || type < 0 || type > 3)
        return -1;
    cplx* ry = make_roots(ny, sign);
    cplx* rz = make_roots(nz, sign);
    cplx* py = (cplx*)malloc(sizeof(cplx) * (size_t)(nk * ny));
    cplx* pz = (cplx*)malloc(sizeof(cplx) * (size_t)(nk * nz));
    if (!ry || !rz || !py || !pz) { free(ry); free(rz); free(py); free(pz); return -2; }
    for (long k = 0; k < nk; ++k) {
        const long ak = ((a[k] % ny) + ny) % ny, bk = ((b[k] % nz) + nz) % nz;
        for (long y = 0; y < ny; ++y) py[k * ny + y] = ry[(ak * y) % ny];
        for (long z = 0; z < nz; ++z) pz[k * nz + z] = rz[(bk * z) % nz];
    }
    psum_ctx base = { nx, ny, z0, z1, chunk, type, NULL, NULL, NULL };
    for (long k = 0; k < nk; ++k) {
        psum_ctx c = base;
        c.py = py + k * ny;
        c.pz = pz + k * nz;
        c.g = g + k * nx;
        parallel_lines(psum_lines, &c, 0, nx, nthreads);
    }
    free(ry); free(rz); free(py); free(pz);
    return 0;
}

/* Full inverse 3D transform: F [nz][ny][H] complex -> f [nz][ny][nx] real.
   F is not modified. */
int p3o_backward(long nx, long ny, long nz, int ty, int tz,
                 const cplx* F, double* f, int nthreads)
{
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    if (ty != P3O_FFT && ty != P3O_EMPTY) return -1;
    if (tz != P3O_FFT && tz != P3O_CHEB && tz != P3O_EMPTY && tz != P3O_SINE) return -1;
    if (tz == P3O_CHEB && nz < 2) return -1;
    long H = nx / 2 + 1;
    size_t cnt = (size_t)H * (size_t)ny * (size_t)nz;
    cplx* w = (cplx*)malloc(sizeof(cplx) * cnt);
    if (!w) return -2;
    memcpy(w, F, sizeof(cplx) * cnt);
    int rc = yz_pass(nx, ny, nz, 2, tz, +1, w, nthreads);
    if (!rc) rc = yz_pass(nx, ny, nz, 1, ty, +1, w, nthreads);
    if (!rc) rc = p3o_x_c2r_rows(nx, w, f, 0, ny * nz, nthreads);
    free(w);
    return rc;
}
