/*
 * bf_oracle.c -- FP64 CPU oracle for the Gauss-polynomial bilateral filter
 * (Chaudhury, "Fast and Accurate Bilateral Filtering using Gauss-Polynomial
 * Decomposition").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline legs of bench.py load this library.  It shares no code, header,
 * table or constant generator with the CUDA library; the product path never
 * calls it.
 *
 * Everything here is plain double-precision C with OpenMP over independent
 * lines or pixels.  No blocking, fusion or reordering beyond what the cited
 * definitions state.
 *
 *   O1  bfo_direct   Eq. (1) with the Gaussian kernels of Eq. (2) on the square
 *                    window [-w, w]^2 of Sec. 1; neighbours that fall outside
 *                    the image are skipped (boundary reading: only in-image
 *                    pixels take part).
 *   O2  bfo_gp       Algorithm 1 (GPF) in Sec. 3, i.e. Eqs. (7)-(11) with the
 *                    centring of Sec. 2 (Proposition / Eq. (6)), using either
 *                      - FIR:  the window sum of Eq. (8), zero extension, or
 *                      - IIR:  Deriche's recursive Gaussian (cited in Sec. 3)
 *                              as the sum of a causal and an anticausal
 *                              recursion on the same input, zero initial
 *                              state at both line ends.
 *   line filters     bfo_line_fir / bfo_line_iir: the 1-D spatial operators
 *                    alone, for pinning them.
 *   bfo_deriche_response: the recursive filter's impulse response h(d).
 *
 * Deriche's 4th-order fit of exp(-x^2/2) (unit sigma) is
 *   h(x) = (a0 cos(w0 x) + a1 sin(w0 x)) e^{-b0 x} + (c0 cos(w1 x) + c1 sin(w1 x)) e^{-b1 x},  x >= 0,
 * with the published constants a0 = 1.680, a1 = 3.735, b0 = 1.783, b1 = 1.723,
 * c0 = -0.6803, c1 = -0.2598, w0 = 0.6318, w1 = 1.997.  At scale sigma, x is
 * replaced by d/sigma for integer lags d.  Writing each term as the real part
 * of a complex exponential gives h(d) = Re[A0 p0^d + A1 p1^d] with
 *   p0 = exp((-b0 + i w0)/sigma), A0 = a0 - i a1,
 *   p1 = exp((-b1 + i w1)/sigma), A1 = c0 - i c1,
 * and the symmetric line operator  y[i] = sum_j h(|i - j|) x[j]  over the
 * in-line samples j is computed by two first-order recursions per pole.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BFO_FIR 1
#define BFO_IIR 2
#define BFO_IIR_ERR 3 /* line filter only: the recursive filter's tap error scale (modal_abs_line) */
#define BFO_BOX 10 /* BFO_BOX + P: P passes of a box of half-width w / P (window of half-width w) */

typedef struct {
    double complex p[2]; /* poles */
    double complex A[2]; /* residues */
} deriche_t;

static void deriche_design(double sigma, deriche_t *D)
{
    const double a0 = 1.680, a1 = 3.735, b0 = 1.783, b1 = 1.723;
    const double c0 = -0.6803, c1 = -0.2598, w0 = 0.6318, w1 = 1.997;
    D->p[0] = cexp((-b0 + I * w0) / sigma);
    D->p[1] = cexp((-b1 + I * w1) / sigma);
    D->A[0] = a0 - I * a1;
    D->A[1] = c0 - I * c1;
}

/* FIR: y[i] = sum_{d=-w..w} taps[|d|] x[i-d], samples outside [0, n) are zero. */
static void fir_line(const double *x, long xs, int n, const double *taps, int w,
                     double *y, long ys)
{
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int d = -w; d <= w; ++d) {
            int j = i - d;
            if (j < 0 || j >= n) continue;
            acc += taps[d < 0 ? -d : d] * x[(long)j * xs];
        }
        y[(long)i * ys] = acc;
    }
}

/* IIR: causal part  sum_{d>=0} h(d) x[i-d]  and anticausal part
 * sum_{d>=1} h(d) x[i+d], both with zero state outside the line. */
static void iir_line(const double *x, long xs, int n, const deriche_t *D,
                     double *y, long ys)
{
    for (int i = 0; i < n; ++i) y[(long)i * ys] = 0.0;
    for (int m = 0; m < 2; ++m) {
        double complex z = 0.0;
        for (int i = 0; i < n; ++i) {
            z = x[(long)i * xs] + D->p[m] * z;
            y[(long)i * ys] += creal(D->A[m] * z);
        }
        double complex v = 0.0;
        for (int i = n - 2; i >= 0; --i) {
            v = D->p[m] * (x[(long)(i + 1) * xs] + v);
            y[(long)i * ys] += creal(D->A[m] * v);
        }
    }
}

/*
 * Error scale of the recursive filter's taps: M(d) = sum_m |A_m| |p_m|^d.  The
 * filter forms h(d) = Re sum_m A_m p_m^d from its modal terms, each carried with
 * a relative error of the order of the arithmetic's, so the error of an
 * effective tap is of the order of eps M(d); in the tail the terms cancel and
 * |h(d)| is far below them.  y[i] = sum_j M(|i - j|) x[j] over the line (zero
 * extension), computed as two first-order recursions per pole with the real
 * factors |p_m|, |A_m| (the same form as iir_line).
 */
static void modal_abs_line(const double *x, long xs, int n, const deriche_t *D, double *y, long ys)
{
    for (int i = 0; i < n; ++i) y[(long)i * ys] = 0.0;
    for (int m = 0; m < 2; ++m) {
        const double r = cabs(D->p[m]), a = cabs(D->A[m]);
        double z = 0.0;
        for (int i = 0; i < n; ++i) {
            z = x[(long)i * xs] + r * z;
            y[(long)i * ys] += a * z;
        }
        double v = 0.0;
        for (int i = n - 2; i >= 0; --i) {
            v = r * (x[(long)(i + 1) * xs] + v);
            y[(long)i * ys] += a * v;
        }
    }
}

/* y[i] = sum_{|d| <= D} a[|d|] x[i - d], zero extension (explicit; a >= 0). */
static void absconv_line(const double *x, long xs, int n, const double *a, int D, double *y, long ys)
{
    for (int i = 0; i < n; ++i) {
        double acc = a[0] * x[(long)i * xs];
        for (int d = 1; d <= D; ++d) {
            if (i - d >= 0) acc += a[d] * x[(long)(i - d) * xs];
            if (i + d < n) acc += a[d] * x[(long)(i + d) * xs];
        }
        y[(long)i * ys] = acc;
    }
}

static void make_taps(double sigma_s, int w, double *taps)
{
    for (int d = 0; d <= w; ++d) taps[d] = exp(-(double)d * d / (2.0 * sigma_s * sigma_s));
}

/*
 * The box-filter variant of the spatial operator (the paper allows any
 * constant-time filter in place of the Gaussian, e.g. a box): P passes of the
 * flat kernel of half-width r, i.e. the P-fold convolution of 2r + 1 ones,
 * half-width w = P r, taps[d] for d = 0..w (symmetric).  Used with the same
 * zero extension of the input as the window sum of Eq. (8).
 */
static void make_box_taps(int passes, int r, double *taps)
{
    const int w = passes * r, n = 2 * w + 1;
    double *k = calloc((size_t)n, sizeof(double)), *t = calloc((size_t)n, sizeof(double));
    for (int i = -r; i <= r; ++i) k[w + i] = 1.0;
    for (int p = 1; p < passes; ++p) {
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = -r; j <= r; ++j)
                if (i - j >= 0 && i - j < n) acc += k[i - j];
            t[i] = acc;
        }
        memcpy(k, t, sizeof(double) * (size_t)n);
    }
    for (int d = 0; d <= w; ++d) taps[d] = k[w + d];
    free(k);
    free(t);
}

int bfo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void bfo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Impulse response of the recursive filter: h[d] for d = 0..n-1. */
void bfo_deriche_response(double sigma, int n, double *h)
{
    deriche_t D;
    deriche_design(sigma, &D);
    for (int d = 0; d < n; ++d) {
        double acc = 0.0;
        for (int m = 0; m < 2; ++m) acc += creal(D.A[m] * cpow(D.p[m], (double)d));
        h[d] = acc;
    }
}

/* Poles and residues as (re, im) pairs: out[0..3] = p0, p1; out[4..7] = A0, A1. */
void bfo_deriche_coefs(double sigma, double *out)
{
    deriche_t D;
    deriche_design(sigma, &D);
    for (int m = 0; m < 2; ++m) {
        out[2 * m] = creal(D.p[m]);
        out[2 * m + 1] = cimag(D.p[m]);
        out[4 + 2 * m] = creal(D.A[m]);
        out[4 + 2 * m + 1] = cimag(D.A[m]);
    }
}

/* 1-D spatial operator on `count` independent lines of length n (row-major). */
void bfo_line_filter(const double *x, int count, int n, double sigma_s, int spatial,
                     int w, double *y)
{
    /* box variant: P passes of a flat kernel, evaluated as its window sum */
    const int box = spatial > BFO_BOX ? spatial - BFO_BOX : 0;
    if (box) spatial = BFO_FIR;
    if (spatial == BFO_FIR) {
        double *taps = malloc(sizeof(double) * (size_t)(w + 1));
        if (box) make_box_taps(box, w / box, taps);
        else make_taps(sigma_s, w, taps);
#pragma omp parallel for schedule(static)
        for (int l = 0; l < count; ++l) fir_line(x + (long)l * n, 1, n, taps, w, y + (long)l * n, 1);
        free(taps);
    } else {
        deriche_t D;
        deriche_design(sigma_s, &D);
        const int err = spatial == BFO_IIR_ERR;
#pragma omp parallel for schedule(static)
        for (int l = 0; l < count; ++l) {
            if (err) modal_abs_line(x + (long)l * n, 1, n, &D, y + (long)l * n, 1);
            else iir_line(x + (long)l * n, 1, n, &D, y + (long)l * n, 1);
        }
    }
}

/*
 * O1 -- direct evaluation of Eq. (1).  Output for the crop rows [r0, r1) and
 * columns [c0, c1) of the H x W image f (row-major, FP64), written densely to
 * out[(r1-r0) x (c1-c0)].  sigma_r = +inf gives the plain normalised spatial
 * filter (range kernel identically one).
 */
void bfo_direct(const double *f, int H, int W, double sigma_s, double sigma_r, int w,
                int r0, int r1, int c0, int c1, double *out)
{
    const int cw = c1 - c0;
    const double inv2s2 = 1.0 / (2.0 * sigma_s * sigma_s);
    const double inv2r2 = isinf(sigma_r) ? 0.0 : 1.0 / (2.0 * sigma_r * sigma_r);
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = r0; y < r1; ++y) {
        for (int x = c0; x < c1; ++x) {
            const double tau = f[(long)y * W + x];
            double num = 0.0, den = 0.0;
            for (int dy = -w; dy <= w; ++dy) {
                const int yy = y - dy;
                if (yy < 0 || yy >= H) continue;
                for (int dx = -w; dx <= w; ++dx) {
                    const int xx = x - dx;
                    if (xx < 0 || xx >= W) continue;
                    const double t = f[(long)yy * W + xx];
                    const double gs = exp(-(double)(dx * dx + dy * dy) * inv2s2);
                    const double gr = exp(-(t - tau) * (t - tau) * inv2r2);
                    num += gs * gr * t;
                    den += gs * gr;
                }
            }
            out[(long)(y - r0) * cw + (x - c0)] = num / den;
        }
    }
}

double bfo_mean(const double *f, long n)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += f[i];
    return s / (double)n;
}

/*
 * Separable spatial operator S applied to the image a, which holds the rows
 * [ylo, yhi) of a W-wide image (row y at a + (y - ylo) * W), evaluated on the crop
 * rows [r0, r1) x columns [c0, c1) into out (dense crop layout).  The row
 * pass filters whole rows; the column pass filters, for each crop column, the
 * rows [ylo, yhi) of the row-filtered image.  For IIR the caller passes
 * ylo = 0, yhi = H so every column is filtered over its full length.
 */
typedef struct {
    int spatial, w;
    const double *taps;
    const deriche_t *D;
    const double *abs_h; /* window taps' error scale, d = 0..abs_D (for kappa; the recursive filter uses modal_abs_line) */
    int abs_D;
} spatial_op;

static void apply_S_impl(const spatial_op *S, int absk, const double *a, int W, int ylo, int yhi,
                         int r0, int r1, int c0, int c1, double *rowtmp, double *out)
{
    const int cw = c1 - c0;
    const int nr = yhi - ylo;
    /* rows: rowtmp[(y - ylo) * cw + (x - c0)] holds the row-filtered image on the crop columns */
#pragma omp parallel
    {
        double *line = malloc(sizeof(double) * (size_t)W);
#pragma omp for schedule(static)
        for (int y = ylo; y < yhi; ++y) {
            const double *src = a + (long)(y - ylo) * W;
            if (absk && S->spatial != BFO_FIR) modal_abs_line(src, 1, W, S->D, line, 1);
            else if (absk) absconv_line(src, 1, W, S->abs_h, S->abs_D < W - 1 ? S->abs_D : W - 1, line, 1);
            else if (S->spatial == BFO_FIR) fir_line(src, 1, W, S->taps, S->w, line, 1);
            else iir_line(src, 1, W, S->D, line, 1);
            memcpy(rowtmp + (long)(y - ylo) * cw, line + c0, sizeof(double) * (size_t)cw);
        }
        free(line);
    }
    /* columns */
#pragma omp parallel
    {
        double *col = malloc(sizeof(double) * (size_t)nr);
#pragma omp for schedule(static)
        for (int x = 0; x < cw; ++x) {
            if (absk && S->spatial != BFO_FIR) modal_abs_line(rowtmp + x, cw, nr, S->D, col, 1);
            else if (absk) absconv_line(rowtmp + x, cw, nr, S->abs_h, S->abs_D < nr - 1 ? S->abs_D : nr - 1, col, 1);
            else if (S->spatial == BFO_FIR) fir_line(rowtmp + x, cw, nr, S->taps, S->w, col, 1);
            else iir_line(rowtmp + x, cw, nr, S->D, col, 1);
            for (int y = r0; y < r1; ++y) out[(long)(y - r0) * cw + x] = col[y - ylo];
        }
        free(col);
    }
}

static void apply_S(const spatial_op *S, const double *a, int W, int ylo, int yhi, int r0, int r1, int c0, int c1,
                    double *rowtmp, double *out)
{
    apply_S_impl(S, 0, a, W, ylo, yhi, r0, r1, c0, c1, rowtmp, out);
}

/*
 * O2 -- Algorithm 1 (GPF).  f is the full H x W image; the result is produced
 * on the crop [r0, r1) x [c0, c1), for each of the nN increasing orders Ns
 * (out and kappa: [nN][crop]; the terms of order N are a prefix of the loop).  t_c: the centre of Sec. 2 (NaN selects the
 * image mean of the algorithm's first step).  spatial: BFO_FIR (window w) or
 * BFO_IIR.  Returns 0 on success, -1 on allocation failure.
 *
 * sigma_r = +inf is taken as its limit: every G_n, n >= 1, vanishes and the
 * result is S(h)/S(1) + t_c, the normalised spatial filter.  Where the
 * denominator Q is not positive, Eq. (11) is undefined and the pixel keeps its
 * own value f (with the window sum this needs odd N, where the truncated
 * exponential has a real root; the recursive filter's small negative tail also
 * does it when (R / sigma_r)^2 is large).
 *
 * lam (may be NULL): a per-pixel factor on the argument of the exponential
 * of Eq. (7), E = exp(-lam h^2 / 2 sigma_r^2) (1 everywhere when NULL); it
 * only serves to pin the sensitivity to that argument (bfo_gp_tangent).
 *
 * kappa (may be NULL): first-order bound on how far relative errors eps in
 * every product entering P and Q (the spatial sums of Eq. (8) and the terms
 * of Eqs. (9)-(10)) can move the result:
 *     kappa = sigma_r (sum_n |G_n| (|h| * |F_{n+1}|) / n! + |P/Q| sum_n |G_n| (|h| * |F_n|) / n!) / |Q|,
 * where |h| * |F| filters |F| with the error scale of the spatial kernel's
 * taps: the window taps themselves, or, for the recursive filter, the
 * magnitude sum_m |A_m| |p_m|^d of its modal terms (modal_abs_line); the
 * result moves by at most about kappa * eps.  The sensitivity to rounding the centred intensity itself is
 * bfo_gp_tangent's.
 * Infinite where Q <= 0.
 */
int bfo_gp(const double *f, int H, int W, double sigma_s, double sigma_r, int nN, const int *Ns,
           double t_c, int spatial, int w, int r0, int r1, int c0, int c1, const double *lam, double *out,
           double *kappa)
{
    /* orders: Ns[0] < Ns[1] < ... ; the loop runs to the last one and the result of each is taken when
       the loop has added its terms (P and Q of order N are the sums over n <= N) */
    if (nN < 1) return -1;
    for (int q = 0; q < nN; ++q)
        if (Ns[q] < 0 || (q > 0 && Ns[q] <= Ns[q - 1])) return -1;
    const int N = Ns[nN - 1];
    /* box variant: P passes of a flat kernel, evaluated as its window sum */
    const int box = spatial > BFO_BOX ? spatial - BFO_BOX : 0;
    if (box) spatial = BFO_FIR;
    const int cw = c1 - c0, ch = r1 - r0;
    const long ncrop = (long)cw * ch;
    int ylo = 0, yhi = H;
    if (spatial == BFO_FIR) {
        ylo = r0 - w < 0 ? 0 : r0 - w;
        yhi = r1 + w > H ? H : r1 + w;
    }
    const long nreg = (long)(yhi - ylo) * W;

    double *taps = NULL;
    deriche_t D;
    spatial_op S = {spatial, w, NULL, NULL, NULL, 0};
    if (spatial == BFO_FIR) {
        taps = malloc(sizeof(double) * (size_t)(w + 1));
        if (!taps) return -1;
        if (box) make_box_taps(box, w / box, taps);
        else make_taps(sigma_s, w, taps);
        S.taps = taps;
    } else {
        deriche_design(sigma_s, &D);
        S.D = &D;
    }
    /* the error scale of each tap for kappa: the window taps (the recursive filter's is modal_abs_line) */
    double *abs_h = NULL;
    if (kappa && spatial == BFO_FIR) {
        abs_h = malloc(sizeof(double) * (size_t)(w + 1));
        if (!abs_h) { free(taps); return -1; }
        for (int d = 0; d <= w; ++d) abs_h[d] = taps[d];
        S.abs_h = abs_h;
        S.abs_D = w;
    }

    /* F and Hs live on the full-width rows [ylo, yhi) (offset so that row y is at (y - ylo) * W) */
    double *F = malloc(sizeof(double) * (size_t)nreg);
    double *Hs = malloc(sizeof(double) * (size_t)nreg);
    double *rowtmp = malloc(sizeof(double) * (size_t)((long)(yhi - ylo) * cw));
    double *Fbar = malloc(sizeof(double) * (size_t)ncrop);
    double *G = malloc(sizeof(double) * (size_t)ncrop);
    double *Hc = malloc(sizeof(double) * (size_t)ncrop);
    double *P = calloc((size_t)ncrop, sizeof(double));
    double *Q = calloc((size_t)ncrop, sizeof(double));
    double *Pa = calloc((size_t)ncrop, sizeof(double));
    double *Qa = calloc((size_t)ncrop, sizeof(double));
    double *Fa = kappa ? malloc(sizeof(double) * (size_t)nreg) : NULL;
    double *FbarA = kappa ? malloc(sizeof(double) * (size_t)ncrop) : NULL;
    if (!F || !Hs || !rowtmp || !Fbar || !G || !Hc || !P || !Q || !Pa || !Qa || (kappa && (!Fa || !FbarA))) {
        free(F); free(Hs); free(rowtmp); free(Fbar); free(G); free(Hc); free(P); free(Q); free(Pa); free(Qa);
        free(Fa); free(FbarA); free(taps); free(abs_h);
        return -1;
    }

    /* step 1: centre */
    if (isnan(t_c)) t_c = bfo_mean(f, (long)H * W);

    if (isinf(sigma_r)) {
        /* limit sigma_r -> inf: numerator S(h), denominator S(1) */
        for (long i = 0; i < nreg; ++i) { F[i] = f[(long)ylo * W + i] - t_c; Hs[i] = 1.0; }
        apply_S(&S, F, W, ylo, yhi, r0, r1, c0, c1, rowtmp, P);
        apply_S(&S, Hs, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Q);
        if (kappa) {
            for (long i = 0; i < nreg; ++i) Fa[i] = fabs(F[i]);
            apply_S_impl(&S, 1, Fa, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Pa);
            apply_S_impl(&S, 1, Hs, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Qa);
        }
        for (int q = 0; q < nN; ++q)
            for (long i = 0; i < ncrop; ++i) {
                out[(long)q * ncrop + i] = P[i] / Q[i] + t_c;
                if (kappa) kappa[(long)q * ncrop + i] = (Pa[i] + fabs(P[i] / Q[i]) * Qa[i]) / fabs(Q[i]);
            }
        goto done;
    }

    /* steps 2, 4, 7 on the rows the operator reads; steps 3, 5, 6 on the crop */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < nreg; ++i) {
        const double h = f[(long)ylo * W + i] - t_c;
        F[i] = exp(-(lam ? lam[(long)ylo * W + i] : 1.0) * h * h / (2.0 * sigma_r * sigma_r));
        Hs[i] = h / sigma_r;
    }
    for (int y = r0; y < r1; ++y)
        for (int x = c0; x < c1; ++x) {
            const long k = (long)(y - r0) * cw + (x - c0);
            Hc[k] = (f[(long)y * W + x] - t_c) / sigma_r;
            G[k] = 1.0;
        }
    /* step 8: filtered F_0 (and, for kappa, the filter of |F_0| with |h|) */
    apply_S(&S, F, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Fbar);
    if (kappa) {
        for (long i = 0; i < nreg; ++i) Fa[i] = fabs(F[i]);
        apply_S_impl(&S, 1, Fa, W, ylo, yhi, r0, r1, c0, c1, rowtmp, FbarA);
    }
    double c = 1.0; /* 1/n! */
    for (int n = 0; n <= N; ++n) {
        /* Eq. (10): Q += G_n Fbar_n / n! */
        for (long i = 0; i < ncrop; ++i) {
            Q[i] += c * G[i] * Fbar[i];
            if (kappa) Qa[i] += fabs(c * G[i]) * FbarA[i];
        }
        /* F_{n+1} = H F_n, then Fbar_{n+1} */
#pragma omp parallel for schedule(static)
        for (long i = 0; i < nreg; ++i) F[i] *= Hs[i];
        apply_S(&S, F, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Fbar);
        if (kappa) {
            for (long i = 0; i < nreg; ++i) Fa[i] = fabs(F[i]);
            apply_S_impl(&S, 1, Fa, W, ylo, yhi, r0, r1, c0, c1, rowtmp, FbarA);
        }
        /* Eq. (9) without the sigma_r factor: P += G_n Fbar_{n+1} / n! */
        for (long i = 0; i < ncrop; ++i) {
            P[i] += c * G[i] * Fbar[i];
            if (kappa) Pa[i] += fabs(c * G[i]) * FbarA[i];
        }
        for (long i = 0; i < ncrop; ++i) G[i] *= Hc[i];
        c /= (double)(n + 1);
        /* step 18 for every requested order n: Eq. (11) with the sigma_r of Eq. (9), then undo the
           centring (Eq. (6)) */
        for (int q = 0; q < nN; ++q) {
            if (Ns[q] != n) continue;
            double *o = out + (long)q * ncrop, *k = kappa ? kappa + (long)q * ncrop : NULL;
            for (long i = 0; i < ncrop; ++i) {
                /* Q <= 0: Eq. (11) is undefined; the pixel keeps its own value */
                const double fi = f[(long)(r0 + i / cw) * W + c0 + i % cw];
                o[i] = Q[i] > 0.0 ? sigma_r * (P[i] / Q[i]) + t_c : fi;
                if (k) k[i] = Q[i] > 0.0 ? sigma_r * (Pa[i] + fabs(P[i] / Q[i]) * Qa[i]) / Q[i] : INFINITY;
            }
        }
    }

done:
    free(F); free(Hs); free(rowtmp); free(Fbar); free(G); free(Hc); free(P); free(Q); free(Pa); free(Qa);
    free(Fa); free(FbarA); free(taps); free(abs_h);
    return 0;
}

/*
 * Joint (cross) bilateral filter, direct: Eq. (1) with the range kernel
 * evaluated on a guide image g instead of f (the extension the paper names in
 * its conclusion): weights g_s(j) g_r(g(i - j) - g(i)), data f(i - j).
 */
void bfo_direct_joint(const double *f, const double *g, int H, int W, double sigma_s, double sigma_r, int w,
                      int r0, int r1, int c0, int c1, double *out)
{
    const int cw = c1 - c0;
    const double inv2s2 = 1.0 / (2.0 * sigma_s * sigma_s);
    const double inv2r2 = isinf(sigma_r) ? 0.0 : 1.0 / (2.0 * sigma_r * sigma_r);
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = r0; y < r1; ++y) {
        for (int x = c0; x < c1; ++x) {
            const double tau = g[(long)y * W + x];
            double num = 0.0, den = 0.0;
            for (int dy = -w; dy <= w; ++dy) {
                const int yy = y - dy;
                if (yy < 0 || yy >= H) continue;
                for (int dx = -w; dx <= w; ++dx) {
                    const int xx = x - dx;
                    if (xx < 0 || xx >= W) continue;
                    const double t = g[(long)yy * W + xx];
                    const double gs = exp(-(double)(dx * dx + dy * dy) * inv2s2);
                    const double gr = exp(-(t - tau) * (t - tau) * inv2r2);
                    num += gs * gr * f[(long)yy * W + xx];
                    den += gs * gr;
                }
            }
            out[(long)(y - r0) * cw + (x - c0)] = num / den;
        }
    }
}

/*
 * Joint (cross) bilateral filter by the Gauss-polynomial decomposition:
 * Algorithm 1 with the range kernel's translate decomposition (Eq. (3)) taken
 * on the centred guide h = g - t_c, so the auxiliary images of Eq. (7) are
 * F_n = H^n exp(-h^2 / 2 sigma_r^2) for the denominator and F_n (f - t_c) for
 * the numerator, n = 0..N (2 (N + 1) filterings):
 *     Q = sum_n G_n S(F_n) / n!,  P = sum_n G_n S(F_n (f - t_c)) / n!,
 *     result = t_c + P / Q,
 * with G_n = H^n at the output pixel (Eqs. (9)-(10) with the data f in place
 * of h in the numerator).  With g = f this is Algorithm 1 (P here is sigma_r
 * times the P of Eq. (9)).  t_c: NaN selects the guide's mean.  Other
 * arguments, lam and kappa as bfo_gp (kappa without the sigma_r factor).
 */
int bfo_gp_joint(const double *f, const double *g, int H, int W, double sigma_s, double sigma_r, int N,
                 double t_c, int spatial, int w, int r0, int r1, int c0, int c1, const double *lam, double *out,
                 double *kappa)
{
    /* box variant: P passes of a flat kernel, evaluated as its window sum */
    const int box = spatial > BFO_BOX ? spatial - BFO_BOX : 0;
    if (box) spatial = BFO_FIR;
    const int cw = c1 - c0, ch = r1 - r0;
    const long ncrop = (long)cw * ch;
    int ylo = 0, yhi = H;
    if (spatial == BFO_FIR) {
        ylo = r0 - w < 0 ? 0 : r0 - w;
        yhi = r1 + w > H ? H : r1 + w;
    }
    const long nreg = (long)(yhi - ylo) * W;

    double *taps = NULL;
    deriche_t D;
    spatial_op S = {spatial, w, NULL, NULL, NULL, 0};
    if (spatial == BFO_FIR) {
        taps = malloc(sizeof(double) * (size_t)(w + 1));
        if (!taps) return -1;
        if (box) make_box_taps(box, w / box, taps);
        else make_taps(sigma_s, w, taps);
        S.taps = taps;
    } else {
        deriche_design(sigma_s, &D);
        S.D = &D;
    }
    double *abs_h = NULL;
    if (kappa && spatial == BFO_FIR) {
        abs_h = malloc(sizeof(double) * (size_t)(w + 1));
        if (!abs_h) { free(taps); return -1; }
        for (int d = 0; d <= w; ++d) abs_h[d] = taps[d];
        S.abs_h = abs_h;
        S.abs_D = w;
    }

    double *F = malloc(sizeof(double) * (size_t)nreg);   /* F_n on the rows the operator reads */
    double *FD = malloc(sizeof(double) * (size_t)nreg);  /* F_n (f - t_c) */
    double *Hs = malloc(sizeof(double) * (size_t)nreg);
    double *Dc = malloc(sizeof(double) * (size_t)nreg);  /* f - t_c */
    double *rowtmp = malloc(sizeof(double) * (size_t)((long)(yhi - ylo) * cw));
    double *Fbar = malloc(sizeof(double) * (size_t)ncrop);
    double *G = malloc(sizeof(double) * (size_t)ncrop);
    double *Hc = malloc(sizeof(double) * (size_t)ncrop);
    double *P = calloc((size_t)ncrop, sizeof(double));
    double *Q = calloc((size_t)ncrop, sizeof(double));
    double *Pa = calloc((size_t)ncrop, sizeof(double));
    double *Qa = calloc((size_t)ncrop, sizeof(double));
    double *Fa = kappa ? malloc(sizeof(double) * (size_t)nreg) : NULL;
    double *FbarA = kappa ? malloc(sizeof(double) * (size_t)ncrop) : NULL;
    if (!F || !FD || !Hs || !Dc || !rowtmp || !Fbar || !G || !Hc || !P || !Q || !Pa || !Qa ||
        (kappa && (!Fa || !FbarA))) {
        free(F); free(FD); free(Hs); free(Dc); free(rowtmp); free(Fbar); free(G); free(Hc); free(P); free(Q);
        free(Pa); free(Qa); free(Fa); free(FbarA); free(taps); free(abs_h);
        return -1;
    }

    /* step 1 on the guide */
    if (isnan(t_c)) t_c = bfo_mean(g, (long)H * W);
    const int inf_r = isinf(sigma_r);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < nreg; ++i) {
        const double h = g[(long)ylo * W + i] - t_c;
        F[i] = inf_r ? 1.0 : exp(-(lam ? lam[(long)ylo * W + i] : 1.0) * h * h / (2.0 * sigma_r * sigma_r));
        Hs[i] = inf_r ? 0.0 : h / sigma_r;
        Dc[i] = f[(long)ylo * W + i] - t_c;
    }
    for (int y = r0; y < r1; ++y)
        for (int x = c0; x < c1; ++x) {
            const long k = (long)(y - r0) * cw + (x - c0);
            Hc[k] = inf_r ? 0.0 : (g[(long)y * W + x] - t_c) / sigma_r;
            G[k] = 1.0;
        }
    double c = 1.0; /* 1/n! */
    const int nmax = inf_r ? 0 : N;
    for (int n = 0; n <= nmax; ++n) {
        if (n > 0) {
#pragma omp parallel for schedule(static)
            for (long i = 0; i < nreg; ++i) F[i] *= Hs[i];
        }
        /* denominator: Q += G_n S(F_n) / n! */
        apply_S(&S, F, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Fbar);
        for (long i = 0; i < ncrop; ++i) Q[i] += c * G[i] * Fbar[i];
        if (kappa) {
            for (long i = 0; i < nreg; ++i) Fa[i] = fabs(F[i]);
            apply_S_impl(&S, 1, Fa, W, ylo, yhi, r0, r1, c0, c1, rowtmp, FbarA);
            for (long i = 0; i < ncrop; ++i) Qa[i] += fabs(c * G[i]) * FbarA[i];
        }
        /* numerator: P += G_n S(F_n (f - t_c)) / n! */
#pragma omp parallel for schedule(static)
        for (long i = 0; i < nreg; ++i) FD[i] = F[i] * Dc[i];
        apply_S(&S, FD, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Fbar);
        for (long i = 0; i < ncrop; ++i) P[i] += c * G[i] * Fbar[i];
        if (kappa) {
            for (long i = 0; i < nreg; ++i) Fa[i] = fabs(FD[i]);
            apply_S_impl(&S, 1, Fa, W, ylo, yhi, r0, r1, c0, c1, rowtmp, FbarA);
            for (long i = 0; i < ncrop; ++i) Pa[i] += fabs(c * G[i]) * FbarA[i];
        }
        for (long i = 0; i < ncrop; ++i) G[i] *= Hc[i];
        c /= (double)(n + 1);
    }
    for (long i = 0; i < ncrop; ++i) {
        /* Q <= 0: the ratio is undefined; the pixel keeps its data value */
        const double fi = f[(long)(r0 + i / cw) * W + c0 + i % cw];
        out[i] = Q[i] > 0.0 ? P[i] / Q[i] + t_c : fi;
        if (kappa) kappa[i] = Q[i] > 0.0 ? (Pa[i] + fabs(P[i] / Q[i]) * Qa[i]) / Q[i] : INFINITY;
    }
    free(F); free(FD); free(Hs); free(Dc); free(rowtmp); free(Fbar); free(G); free(Hc); free(P); free(Q);
    free(Pa); free(Qa); free(Fa); free(FbarA); free(taps); free(abs_h);
    return 0;
}

/*
 * Probe signs for bfo_gp_tangent: the top bit of splitmix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", 2014) applied to
 * the seed mixed with a per-pixel counter.
 */
static unsigned long long bfo_splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double bfo_probe_sign(unsigned long long seed, long counter)
{
    return (bfo_splitmix64(seed ^ bfo_splitmix64((unsigned long long)counter)) >> 63) ? -1.0 : 1.0;
}

/* the sign bfo_gp_tangent draws for pixel index y W + x, component k (0: delta, 1: eta, 2: xi) */
double bfo_gp_probe_sign(unsigned long long seed, long pixel, int k)
{
    return bfo_probe_sign(seed, 3 * pixel + k);
}

/*
 * First-order change of O2 (bfo_gp; with a guide g: bfo_gp_joint) on the crop
 * under relative perturbations, at every pixel j of the image, of
 *   delta_j: the centred intensity H_j = (g_j - t_c) / sigma_r (g = f for the
 *            plain filter) in all its uses: the exponential and the power of
 *            Eq. (7) where j is an input, G_n = H^n where j is the output pixel;
 *   eta_j:   the argument lam_j H_j^2 / 2 of the exponential of Eq. (7) alone;
 *   xi_j:    the centred data f_j - t_c (joint filter only).
 * This is the derivative of Eqs. (7)-(11), taken in forward mode:
 *   dF_n = F_n ((n - lam H^2) delta - lam (H^2 / 2) eta),   dG_n = n G_n delta,
 *   dQ = sum_n (dG_n S F_n + G_n S dF_n) / n!,   dP the same with F_{n+1}
 *   (joint: with F_n (f - t_c), whose change also has F_n (f - t_c) xi),
 *   dy = sigma_r (dP - (P / Q) dQ) / Q   (joint: without sigma_r),
 * and for sigma_r = inf (y = S(h) / S(1) + t_c)  dy = S(h delta) / S(1)
 * (joint: S((f - t_c) xi) / S(1)).
 * npr probes: either one explicit probe (delta, eta, xi are [H][W] arrays or
 * NULL for zero; spec unused) or, when all three are NULL, npr drawn ones:
 * spec[7p .. 7p+6] = {d0, d1, e0, e1, x0, x1, seed} gives delta_j = d0 + d1 s_j,
 * eta_j = e0 + e1 s'_j, xi_j = x0 + x1 s''_j with the signs of
 * bfo_gp_probe_sign(seed, y W + x, 0 / 1 / 2).  dy: [npr][nN][crop] for the
 * increasing orders Ns; where Q <= 0
 * (the pixel keeps its value) the change of that value.  t_c: NaN selects the
 * mean (of g for the joint filter).  Returns 0,
 * or -1 on allocation failure or bad arguments.
 */
int bfo_gp_tangent(const double *f, const double *g, int H, int W, double sigma_s, double sigma_r, int nN,
                   const int *Ns, double t_c, int spatial, int w, int r0, int r1, int c0, int c1, const double *lam,
                   int npr, const double *spec, const double *delta, const double *eta, const double *xi, double *dy)
{
    if (nN < 1) return -1;
    for (int q = 0; q < nN; ++q)
        if (Ns[q] < 0 || (q > 0 && Ns[q] <= Ns[q - 1])) return -1;
    const int N = Ns[nN - 1];
    const int joint = g != NULL;
    const int explicit_probe = delta || eta || xi;
    if (npr < 1 || (explicit_probe && npr != 1) || (!explicit_probe && !spec)) return -1;
    const int box = spatial > BFO_BOX ? spatial - BFO_BOX : 0;
    if (box) spatial = BFO_FIR;
    const int cw = c1 - c0, ch = r1 - r0;
    const long ncrop = (long)cw * ch;
    int ylo = 0, yhi = H;
    if (spatial == BFO_FIR) {
        ylo = r0 - w < 0 ? 0 : r0 - w;
        yhi = r1 + w > H ? H : r1 + w;
    }
    const long nreg = (long)(yhi - ylo) * W;
    const int inf_r = isinf(sigma_r);
    /* channels: F_n, n = 0..N+1 (plain); F_n and F_n (f - t_c), n = 0..N (joint) */
    const int K = joint ? 2 * (N + 1) : (inf_r ? 2 : N + 2);

    double *taps = NULL;
    deriche_t D;
    spatial_op S = {spatial, w, NULL, NULL, NULL, 0};
    if (spatial == BFO_FIR) {
        taps = malloc(sizeof(double) * (size_t)(w + 1));
        if (!taps) return -1;
        if (box) make_box_taps(box, w / box, taps);
        else make_taps(sigma_s, w, taps);
        S.taps = taps;
    } else {
        deriche_design(sigma_s, &D);
        S.D = &D;
    }
    double *E = malloc(sizeof(double) * (size_t)nreg);      /* exp(-lam H^2 / 2) */
    double *Hs = malloc(sizeof(double) * (size_t)nreg);     /* H on the operator's rows */
    double *L2 = malloc(sizeof(double) * (size_t)nreg);     /* lam H^2 */
    double *Dc = malloc(sizeof(double) * (size_t)nreg);     /* f - t_c */
    double *Fn = malloc(sizeof(double) * (size_t)nreg);
    double *dF = malloc(sizeof(double) * (size_t)nreg);
    double *pd = malloc(sizeof(double) * (size_t)nreg);     /* the probe's delta, eta, xi on the rows */
    double *pe = malloc(sizeof(double) * (size_t)nreg);
    double *px = malloc(sizeof(double) * (size_t)nreg);
    double *rowtmp = malloc(sizeof(double) * (size_t)((long)(yhi - ylo) * cw));
    double *Fb = malloc(sizeof(double) * (size_t)ncrop * K);  /* S of every channel on the crop */
    double *dFb = malloc(sizeof(double) * (size_t)ncrop);
    double *Hc = malloc(sizeof(double) * (size_t)ncrop);
    double *P = calloc((size_t)ncrop * nN, sizeof(double)); /* [order][crop] */
    double *Q = calloc((size_t)ncrop * nN, sizeof(double));
    double *dP = malloc(sizeof(double) * (size_t)ncrop * nN);
    double *dQ = malloc(sizeof(double) * (size_t)ncrop * nN);
    double *Gc = malloc(sizeof(double) * (size_t)ncrop);
    double *dc = malloc(sizeof(double) * (size_t)ncrop);    /* delta at the crop's output pixels */
    double *Wp = malloc(sizeof(double) * (size_t)ncrop);
    int rc = -1;
    if (!E || !Hs || !L2 || !Dc || !Fn || !dF || !pd || !pe || !px || !rowtmp || !Fb || !dFb || !Hc || !P || !Q ||
        !dP || !dQ || !Gc || !dc || !Wp)
        goto out;
    rc = 0;
    const double *rng_src = joint ? g : f;
    if (isnan(t_c)) t_c = bfo_mean(rng_src, (long)H * W);
    for (long i = 0; i < nreg; ++i) {
        const double h = rng_src[(long)ylo * W + i] - t_c;
        const double l = lam ? lam[(long)ylo * W + i] : 1.0;
        Hs[i] = inf_r ? 0.0 : h / sigma_r;
        L2[i] = l * Hs[i] * Hs[i];
        E[i] = exp(-0.5 * L2[i]);
        Dc[i] = (joint ? f[(long)ylo * W + i] : rng_src[(long)ylo * W + i]) - t_c;
    }
    for (int y = r0; y < r1; ++y)
        for (int x = c0; x < c1; ++x)
            Hc[(long)(y - r0) * cw + (x - c0)] = inf_r ? 0.0 : (rng_src[(long)y * W + x] - t_c) / sigma_r;

    /* forward: every filtered channel on the crop (Fb), then P and Q */
    if (!joint && inf_r) {
        /* plain filter, sigma_r = inf: channel 0 = 1, channel 1 = h */
        for (long i = 0; i < nreg; ++i) Fn[i] = 1.0;
        apply_S(&S, Fn, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Fb);
        apply_S(&S, Dc, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Fb + ncrop);
        for (int q = 0; q < nN; ++q)
            for (long i = 0; i < ncrop; ++i) {
                Q[(long)q * ncrop + i] = Fb[i];
                P[(long)q * ncrop + i] = Fb[ncrop + i];
            }
    } else {
        for (long i = 0; i < nreg; ++i) Fn[i] = E[i];
        const int nch = joint ? N + 1 : N + 2; /* powers n = 0..nch-1 */
        for (int n = 0; n < nch; ++n) {
            if (n > 0)
                for (long i = 0; i < nreg; ++i) Fn[i] *= Hs[i];
            if (joint) {
                apply_S(&S, Fn, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Fb + (long)(2 * n) * ncrop);
                for (long i = 0; i < nreg; ++i) dF[i] = Fn[i] * Dc[i];
                apply_S(&S, dF, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Fb + (long)(2 * n + 1) * ncrop);
            } else {
                apply_S(&S, Fn, W, ylo, yhi, r0, r1, c0, c1, rowtmp, Fb + (long)n * ncrop);
            }
        }
        /* Eqs. (9)-(10): Q = sum_{n<=N} G_n Fbar_n / n!, P = sum_{n<=N} G_n Fbar_{n+1} / n!
           (joint: P with the data channel of power n) */
        for (long i = 0; i < ncrop; ++i) {
            double gn = 1.0, c = 1.0, sq = 0.0, spp = 0.0;
            for (int n = 0, q = 0; n <= N; ++n) {
                if (joint) {
                    sq += c * gn * Fb[(long)(2 * n) * ncrop + i];
                    spp += c * gn * Fb[(long)(2 * n + 1) * ncrop + i];
                } else {
                    sq += c * gn * Fb[(long)n * ncrop + i];
                    spp += c * gn * Fb[(long)(n + 1) * ncrop + i];
                }
                if (n == Ns[q]) {
                    Q[(long)q * ncrop + i] = sq;
                    P[(long)q * ncrop + i] = spp;
                    ++q;
                }
                gn *= Hc[i];
                c /= (double)(n + 1);
            }
        }
    }

    /* probes */
    for (int p = 0; p < npr; ++p) {
        const double *sp = spec ? spec + 7 * p : NULL;
        const unsigned long long seed = sp ? (unsigned long long)sp[6] : 0ull;
        for (int y = ylo; y < yhi; ++y)
            for (int x = 0; x < W; ++x) {
                const long j = (long)y * W + x, i = (long)(y - ylo) * W + x;
                if (explicit_probe) {
                    pd[i] = delta ? delta[j] : 0.0;
                    pe[i] = eta ? eta[j] : 0.0;
                    px[i] = xi ? xi[j] : 0.0;
                } else {
                    pd[i] = sp[0] + sp[1] * bfo_gp_probe_sign(seed, j, 0);
                    pe[i] = sp[2] + sp[3] * bfo_gp_probe_sign(seed, j, 1);
                    px[i] = sp[4] + sp[5] * bfo_gp_probe_sign(seed, j, 2);
                }
            }
        for (int y = r0; y < r1; ++y)
            for (int x = c0; x < c1; ++x)
                dc[(long)(y - r0) * cw + (x - c0)] = pd[(long)(y - ylo) * W + x];
        double *out = dy + (long)p * nN * ncrop;
        if (!joint && inf_r) {
            /* dy = S(h delta) / S(1), the same for every order */
            for (long i = 0; i < nreg; ++i) dF[i] = Dc[i] * pd[i];
            apply_S(&S, dF, W, ylo, yhi, r0, r1, c0, c1, rowtmp, dFb);
            for (int q = 0; q < nN; ++q)
                for (long i = 0; i < ncrop; ++i) out[(long)q * ncrop + i] = dFb[i] / Q[i];
            continue;
        }
        /* output-pixel part: dG_n = n G_n delta */
        for (long i = 0; i < ncrop; ++i) {
            double gn = 1.0, c = 1.0, sq = 0.0, spp = 0.0;
            for (int n = 0, q = 0; n <= N; ++n) {
                if (joint) {
                    sq += c * n * gn * Fb[(long)(2 * n) * ncrop + i];
                    spp += c * n * gn * Fb[(long)(2 * n + 1) * ncrop + i];
                } else {
                    sq += c * n * gn * Fb[(long)n * ncrop + i];
                    spp += c * n * gn * Fb[(long)(n + 1) * ncrop + i];
                }
                if (n == Ns[q]) {
                    dQ[(long)q * ncrop + i] = sq * dc[i];
                    dP[(long)q * ncrop + i] = spp * dc[i];
                    ++q;
                }
                gn *= Hc[i];
                c /= (double)(n + 1);
            }
        }
        /* input part: dF_n = F_n ((n - lam H^2) delta - lam (H^2 / 2) eta), filtered; channel n enters Q
           with weight G_n / n! (n <= N) and P with G_{n-1} / (n-1)! (n >= 1; joint: its data channel, G_n / n!) */
        for (long i = 0; i < nreg; ++i) Fn[i] = E[i];
        for (long i = 0; i < ncrop; ++i) {
            Gc[i] = 1.0; /* G_n / n! */
            Wp[i] = 0.0; /* G_{n-1} / (n-1)! */
        }
        const int nch = joint ? N + 1 : N + 2;
        for (int n = 0; n < nch; ++n) {
            if (n > 0)
                for (long i = 0; i < nreg; ++i) Fn[i] *= Hs[i];
            for (long i = 0; i < nreg; ++i) dF[i] = Fn[i] * ((n - L2[i]) * pd[i] - 0.5 * L2[i] * pe[i]);
            apply_S(&S, dF, W, ylo, yhi, r0, r1, c0, c1, rowtmp, dFb);
            /* order N takes channel n into Q when n <= N and into P when n <= N + 1 (joint: n <= N) */
            for (int q = 0; q < nN; ++q) {
                double *dq = dQ + (long)q * ncrop, *dp = dP + (long)q * ncrop;
                for (long i = 0; i < ncrop; ++i) {
                    if (n <= Ns[q]) dq[i] += Gc[i] * dFb[i];
                    if (!joint && n >= 1 && n <= Ns[q] + 1) dp[i] += Wp[i] * dFb[i];
                }
            }
            if (joint) {
                /* data channel F_n (f - t_c): the same change times (f - t_c), plus F_n (f - t_c) xi */
                for (long i = 0; i < nreg; ++i) dF[i] = (dF[i] + Fn[i] * px[i]) * Dc[i];
                apply_S(&S, dF, W, ylo, yhi, r0, r1, c0, c1, rowtmp, dFb);
                for (int q = 0; q < nN; ++q)
                    if (n <= Ns[q])
                        for (long i = 0; i < ncrop; ++i) dP[(long)q * ncrop + i] += Gc[i] * dFb[i];
            }
            for (long i = 0; i < ncrop; ++i) {
                Wp[i] = Gc[i];
                Gc[i] *= Hc[i] / (double)(n + 1);
            }
        }
        const double pref = joint ? 1.0 : sigma_r;
        for (long e = 0; e < (long)nN * ncrop; ++e) {
            /* Q <= 0: y is the pixel's own (data) value, which moves with its own perturbation */
            const long i = e % ncrop;
            const long j = (long)(r0 + i / cw - ylo) * W + c0 + i % cw;
            out[e] = Q[e] > 0.0 ? pref * (dP[e] - (P[e] / Q[e]) * dQ[e]) / Q[e] : Dc[j] * (joint ? px[j] : pd[j]);
        }
    }
out:
    free(taps); free(E); free(Hs); free(L2); free(Dc); free(Fn); free(dF); free(pd); free(pe); free(px);
    free(rowtmp); free(Fb); free(dFb); free(Hc); free(P); free(Q); free(dP); free(dQ); free(Gc); free(dc);
    free(Wp);
    return rc;
}

/*
 * Eq. (5): the Gauss-polynomial of degree N that replaces the translated range
 * kernel g_{sigma_r}(t - tau) of Eq. (3): the two Gaussian factors times the
 * first N + 1 Taylor terms of exp(tau t / sigma_r^2) (Eq. (4)).
 */
double bfo_gp_kernel(double t, double tau, double sigma_r, int N)
{
    const double x = tau * t / (sigma_r * sigma_r);
    double term = 1.0, sum = 0.0;
    for (int n = 0; n <= N; ++n) {
        sum += term;
        term *= x / (double)(n + 1);
    }
    return exp(-tau * tau / (2.0 * sigma_r * sigma_r)) * exp(-t * t / (2.0 * sigma_r * sigma_r)) * sum;
}

/*
 * O3 -- reverse-mode derivative of O2 (Algorithm 1) on the full image, in the
 * paper's own variables.  With H = h / sigma_r, E = exp(-h^2 / 2 sigma_r^2),
 * G_n = H^n, F_n = E H^n, Fbar_n = S F_n, c_n = 1/n!:
 *     P = sum_{n<=N} c_n G_n Fbar_{n+1},  Q = sum_{n<=N} c_n G_n Fbar_n,
 *     y = sigma_r P / Q + t_c   (Eqs. (9)-(11), Eq. (6)).
 * Given ybar = dL/dy, with Pbar = ybar sigma_r / Q and Qbar = -ybar sigma_r P / Q^2:
 *   direct:   Hbar_i = sum_n c_n n H_i^{n-1} (Pbar_i Fbar_{n+1} + Qbar_i Fbar_n)
 *   through S (S is symmetric, so its adjoint is S itself):
 *             lambda_k = Pbar c_{k-1} G_{k-1} [k >= 1] + Qbar c_k G_k [k <= N],  mu_k = S lambda_k,
 *             dF_k/dh = E (k H^{k-1} / sigma_r - h H^k / sigma_r^2)
 *   hbar = sum_k mu_k dF_k/dh + Hbar / sigma_r,
 *   fbar = hbar + (sum ybar - sum hbar) / |I|  when t_c is the mean (Algorithm 1, step 1),
 *          hbar                                 when t_c is given.
 *   sigma_r: y depends on it through the explicit factor, H (dH/dsigma_r = -H/sigma_r)
 *   and E (dE/dsigma_r = E h^2 / sigma_r^3).
 *   A pixel whose Q <= 0 keeps its value (y = f): it passes ybar to its own input only.
 * Full image only (no crop).  Returns 0, or -1 on allocation failure.
 */
int bfo_gp_adjoint(const double *f, int H_, int W, double sigma_s, double sigma_r, int N, double t_c_given,
                   int spatial, int w, const double *ybar, double *fbar, double *sigma_r_bar)
{
    /* box variant: P passes of a flat kernel, evaluated as its window sum */
    const int box = spatial > BFO_BOX ? spatial - BFO_BOX : 0;
    if (box) spatial = BFO_FIR;
    const long n = (long)H_ * W;
    const int K = N + 2;
    double *taps = NULL;
    deriche_t D;
    spatial_op S = {spatial, w, NULL, NULL, NULL, 0};
    if (spatial == BFO_FIR) {
        taps = malloc(sizeof(double) * (size_t)(w + 1));
        if (!taps) return -1;
        if (box) make_box_taps(box, w / box, taps);
        else make_taps(sigma_s, w, taps);
        S.taps = taps;
    } else {
        deriche_design(sigma_s, &D);
        S.D = &D;
    }
    double *h = malloc(sizeof(double) * (size_t)n);
    double *Hh = malloc(sizeof(double) * (size_t)n);
    double *E = malloc(sizeof(double) * (size_t)n);
    double *Fb = malloc(sizeof(double) * (size_t)n * K);   /* Fbar_k, k = 0..N+1 */
    double *tmp = malloc(sizeof(double) * (size_t)n);
    double *rowtmp = malloc(sizeof(double) * (size_t)n);
    double *P = calloc((size_t)n, sizeof(double));
    double *Q = calloc((size_t)n, sizeof(double));
    double *Pb = malloc(sizeof(double) * (size_t)n);
    double *Qb = malloc(sizeof(double) * (size_t)n);
    double *hb = calloc((size_t)n, sizeof(double));
    double *lam = malloc(sizeof(double) * (size_t)n);
    double *mu = malloc(sizeof(double) * (size_t)n);
    if (!h || !Hh || !E || !Fb || !tmp || !rowtmp || !P || !Q || !Pb || !Qb || !hb || !lam || !mu) {
        free(h); free(Hh); free(E); free(Fb); free(tmp); free(rowtmp); free(P); free(Q); free(Pb); free(Qb);
        free(hb); free(lam); free(mu); free(taps);
        return -1;
    }
    const int centre_mean = isnan(t_c_given);
    const double t_c = centre_mean ? bfo_mean(f, n) : t_c_given;
    for (long i = 0; i < n; ++i) {
        h[i] = f[i] - t_c;
        Hh[i] = h[i] / sigma_r;
        E[i] = exp(-h[i] * h[i] / (2.0 * sigma_r * sigma_r));
    }
    /* forward: Fbar_k = S(E H^k) for k = 0..N+1 */
    for (long i = 0; i < n; ++i) tmp[i] = E[i];
    for (int k = 0; k < K; ++k) {
        apply_S(&S, tmp, W, 0, H_, 0, H_, 0, W, rowtmp, Fb + (long)k * n);
        for (long i = 0; i < n; ++i) tmp[i] *= Hh[i];
    }
    double sr_bar = 0.0;
    for (long i = 0; i < n; ++i) {
        double g = 1.0, c = 1.0;
        for (int k = 0; k <= N; ++k) {
            P[i] += c * g * Fb[(long)(k + 1) * n + i];
            Q[i] += c * g * Fb[(long)k * n + i];
            g *= Hh[i];
            c /= (double)(k + 1);
        }
        if (!(Q[i] > 0.0)) {
            /* Q <= 0: y = f (the pixel keeps its value), so dL/df gets ybar directly; written as
               y = t_c + h, its t_c part cancels in the centring term below */
            Pb[i] = Qb[i] = 0.0;
            hb[i] += ybar[i];
            continue;
        }
        Pb[i] = ybar[i] * sigma_r / Q[i];
        Qb[i] = -ybar[i] * sigma_r * P[i] / (Q[i] * Q[i]);
        sr_bar += ybar[i] * P[i] / Q[i]; /* explicit sigma_r factor */
        /* direct dependence on H_i through G_n(i) */
        double Hbar = 0.0, Gsr = 0.0, gm1 = 0.0; /* gm1 = H^{n-1} */
        c = 1.0;
        g = 1.0;
        for (int k = 0; k <= N; ++k) {
            const double term = Pb[i] * Fb[(long)(k + 1) * n + i] + Qb[i] * Fb[(long)k * n + i];
            if (k >= 1) Hbar += c * k * gm1 * term;
            Gsr += c * (-(double)k / sigma_r) * g * term; /* dG_k/dsigma_r = -k G_k / sigma_r */
            gm1 = g;
            g *= Hh[i];
            c /= (double)(k + 1);
        }
        hb[i] += Hbar / sigma_r;
        sr_bar += Gsr;
    }
    /* through S: lambda_k, mu_k = S lambda_k, then dF_k/dh and dF_k/dsigma_r */
    double c_k = 1.0;          /* 1/k! */
    double c_km1 = 0.0;        /* 1/(k-1)! */
    for (int k = 0; k < K; ++k) {
        for (long i = 0; i < n; ++i) {
            double l = 0.0;
            const double Gk = pow(Hh[i], (double)k);
            if (k >= 1) l += Pb[i] * c_km1 * pow(Hh[i], (double)(k - 1));
            if (k <= N) l += Qb[i] * c_k * Gk;
            lam[i] = l;
        }
        apply_S(&S, lam, W, 0, H_, 0, H_, 0, W, rowtmp, mu);
        for (long i = 0; i < n; ++i) {
            const double Hk = pow(Hh[i], (double)k);
            const double Hkm1 = k >= 1 ? pow(Hh[i], (double)(k - 1)) : 0.0;
            const double dFdh = E[i] * ((double)k * Hkm1 / sigma_r - h[i] * Hk / (sigma_r * sigma_r));
            hb[i] += mu[i] * dFdh;
            const double Fk = E[i] * Hk;
            sr_bar += mu[i] * Fk * (h[i] * h[i] / (sigma_r * sigma_r * sigma_r) - (double)k / sigma_r);
        }
        c_km1 = c_k;
        c_k /= (double)(k + 1);
    }
    double sy = 0.0, sh = 0.0;
    for (long i = 0; i < n; ++i) {
        sy += ybar[i];
        sh += hb[i];
    }
    for (long i = 0; i < n; ++i) fbar[i] = hb[i] + (centre_mean ? (sy - sh) / (double)n : 0.0);
    *sigma_r_bar = sr_bar;
    free(h); free(Hh); free(E); free(Fb); free(tmp); free(rowtmp); free(P); free(Q); free(Pb); free(Qb);
    free(hb); free(lam); free(mu); free(taps);
    return 0;
}
