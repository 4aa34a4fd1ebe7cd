/*
 * anova_oracle.c -- plain FP64 CPU oracle for the ANOVA-Gaussian fast summation
 * of Nestler, Stoll and Wagner, "Learning in High-Dimensional Feature Spaces
 * Using ANOVA-Based Fast Matrix-Vector Multiplication" (arXiv 2111.10140).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the test suite, the package
 * smoke check and the benchmark's CPU-baseline leg load it; the product path
 * never does.  It shares no code, header, table or helper with the CUDA path.
 *
 * Every routine follows the paper's formulas in the paper's order:
 *   O1  direct ANOVA-Gaussian matrix-vector product
 *         Sec. 2, Eq. (mult_with_K); Sec. 3, Eq. (extended_Gaussian_ANOVA_kernel)
 *   O2  fast summation  s = Phi_z D Phi^* alpha  per window
 *         Sec. 4.1, Eq. (nfft) and Eq. (adjnfft); Sec. 4.2, Eq. (kernelapprox)
 *         and Eq. (fastsum); Sec. 4.3; windows and weights, Sec. 5
 *   O3  conjugate gradients on (K + lambda I) alpha = y, Sec. 2
 *   O4  brute-force NDFT and adjoint NDFT, Eq. (nfft) and Eq. (adjnfft)
 *
 * Readings where the paper is silent (it leaves the NFFT window, cutoff,
 * oversampling and the regularisation constants to the cited NFFT papers):
 *   - Kaiser-Bessel window in grid units t:
 *       phi(t) = sinh(b sqrt(m^2 - t^2)) / (pi sqrt(m^2 - t^2)),  |t| <= m,
 *     value b/pi at |t| = m, 0 beyond; b = pi (2 - 1/sigma).  Its Fourier
 *     transform at frequency k of an n_os grid is I0(m sqrt(b^2 - (2 pi k/n_os)^2)).
 *   - taps per dimension: u = floor(n_os x) - m ... floor(n_os x) + m + 1.
 *   - nodes are scaled per window into the ball of radius 1/4 - epsB/2 around
 *     the bounding-box midpoint (the "h^{-1} x" scaling of Sec. 4.2); the
 *     kernel width scales with them.
 *   - the regularised kernel is the Gaussian for r <= 1/2 - epsB, a two-point
 *     Taylor polynomial of degree 2p-1 on (1/2 - epsB, 1/2] that ends at the
 *     constant K(1/2) with vanishing derivatives, and K(1/2) beyond (Sec. 4.2,
 *     radial truncation as in the fastsum figure caption).
 *   - grid and frequency arrays are stored with the centred index of the
 *     paper's I_M: value v in {-M/2..M/2-1} sits at position v + M/2.
 *
 * All arithmetic is FP64.  OpenMP only splits independent outer loops.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* small helpers                                                              */
/* ------------------------------------------------------------------------ */

static int win_dim(const int *w)
{
    int d = 0;
    while (d < 3 && w[d] >= 0) d++;
    return d;
}

/* wrap an integer grid value into {-M/2 .. M/2-1} and return its centred position */
static long centred_pos(long v, long M)
{
    long r = v % M;
    if (r < 0) r += M;            /* r in [0, M) */
    if (r >= M / 2) r -= M;       /* value in [-M/2, M/2) */
    return r + M / 2;
}

static long ipow(long a, int e)
{
    long r = 1;
    while (e-- > 0) r *= a;
    return r;
}

/* ------------------------------------------------------------------------ */
/* O1: direct sum, Sec. 2 Eq. (mult_with_K) with the kernel of Sec. 3.       */
/*   out_i = sum_l eta_l sum_j alpha_j exp(-||z_i^{W_l} - x_j^{W_l}||^2/ell^2) */
/* Z may equal X (the kernel-matrix product) or hold test points (Eq. kernelsum). */
/* ------------------------------------------------------------------------ */
void orc_direct(const double *Z, long Nz, long ldz,
                const double *X, long Nx, long ldx,
                const int *win, int P, const double *eta, double ell,
                const double *alpha, double *out)
{
    const double inv_ell2 = 1.0 / (ell * ell);
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < Nz; i++) {
        double acc = 0.0;
        for (int l = 0; l < P; l++) {
            const int *w = win + 3 * l;
            int dA = win_dim(w);
            double sl = 0.0;
            for (long j = 0; j < Nx; j++) {
                double r2 = 0.0;
                for (int t = 0; t < dA; t++) {
                    double df = Z[i * ldz + w[t]] - X[j * ldx + w[t]];
                    r2 += df * df;
                }
                sl += alpha[j] * exp(-r2 * inv_ell2);
            }
            acc += eta[l] * sl;
        }
        out[i] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Node scaling (Sec. 4.2: scaled nodes h^{-1} x on the torus T^d).          */
/* centre = midpoint of the bounding box of the window's coordinates over    */
/* the given point sets; s = RB / max ||x - centre||.  When every point      */
/* coincides the scale is 1.                                                  */
/* ------------------------------------------------------------------------ */
void orc_window_frame(const double *X, long Nx, long ldx,
                      const double *Z, long Nz, long ldz,
                      const int *w, double RB, double *centre, double *scale)
{
    int dA = win_dim(w);
    for (int t = 0; t < 3; t++) centre[t] = 0.0;
    for (int t = 0; t < dA; t++) {
        double lo = INFINITY, hi = -INFINITY;
        for (long j = 0; j < Nx; j++) {
            double v = X[j * ldx + w[t]];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        for (long j = 0; j < Nz; j++) {
            double v = Z[j * ldz + w[t]];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        centre[t] = 0.5 * (lo + hi);
    }
    double rmax = 0.0;
    for (long j = 0; j < Nx; j++) {
        double r2 = 0.0;
        for (int t = 0; t < dA; t++) {
            double df = X[j * ldx + w[t]] - centre[t];
            r2 += df * df;
        }
        if (r2 > rmax) rmax = r2;
    }
    for (long j = 0; j < Nz; j++) {
        double r2 = 0.0;
        for (int t = 0; t < dA; t++) {
            double df = Z[j * ldz + w[t]] - centre[t];
            r2 += df * df;
        }
        if (r2 > rmax) rmax = r2;
    }
    rmax = sqrt(rmax);
    *scale = (rmax > 0.0) ? RB / rmax : 1.0;
}

/* ------------------------------------------------------------------------ */
/* Kaiser-Bessel window and its Fourier transform (NFFT parameters that      */
/* Sec. 4.1 leaves to the cited NFFT3 paper).                                 */
/* ------------------------------------------------------------------------ */
double orc_bessel_i0(double x)
{
    /* power series sum_k ((x/2)^k / k!)^2, summed until the terms vanish */
    double q = 0.25 * x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; k++) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

double orc_kb_phi(double t, int m, double b)
{
    double at = fabs(t);
    if (at > (double)m) return 0.0;
    double s = sqrt((double)m * m - t * t);
    if (s == 0.0) return b / M_PI;
    return sinh(b * s) / (M_PI * s);
}

double orc_kb_phihat(long k, long nos, int m, double b)
{
    double w = 2.0 * M_PI * (double)k / (double)nos;
    return orc_bessel_i0((double)m * sqrt(b * b - w * w));
}

/* ------------------------------------------------------------------------ */
/* Regularised kernel K_R(r) (Sec. 4.2, periodisation with a smooth          */
/* polynomial transition, radially truncated in several dimensions).          */
/* ------------------------------------------------------------------------ */

/* j-th derivative of exp(-r^2/ell^2):  (-1/ell)^j H_j(r/ell) exp(-r^2/ell^2) */
double orc_gauss_deriv(int j, double r, double ell)
{
    double x = r / ell;
    double hm = 1.0, h = 2.0 * x;          /* H_0, H_1 (physicists') */
    double Hj;
    if (j == 0) Hj = 1.0;
    else if (j == 1) Hj = h;
    else {
        for (int i = 1; i < j; i++) {
            double hn = 2.0 * x * h - 2.0 * (double)i * hm;
            hm = h;
            h = hn;
        }
        Hj = h;
    }
    double sgn = (j % 2) ? -1.0 : 1.0;
    return sgn * pow(ell, -(double)j) * Hj * exp(-x * x);
}

static double binom(int nn, int kk)
{
    double r = 1.0;
    for (int i = 1; i <= kk; i++) r = r * (double)(nn - kk + i) / (double)i;
    return r;
}

/* two-point Taylor polynomial of degree 2p-1 on [a, e]: matches f^{(j)}(a)
 * and f^{(j)}(e) = c delta_{j0} for j = 0..p-1 */
double orc_two_point_taylor(double r, double a, double e, int p, double ell, double c)
{
    double L = e - a;
    double ua = (r - a) / L, ue = (e - r) / L;
    double sum = 0.0, fact = 1.0;
    for (int j = 0; j < p; j++) {
        if (j > 0) fact *= (double)j;
        double inner_a = 0.0, inner_e = 0.0;
        for (int q = 0; q <= p - 1 - j; q++) {
            double cq = binom(p - 1 + q, q);
            inner_a += cq * pow(ua, (double)q);
            inner_e += cq * pow(ue, (double)q);
        }
        double fa = orc_gauss_deriv(j, a, ell);
        double fe = (j == 0) ? c : 0.0;
        sum += fa * pow(r - a, (double)j) / fact * pow(ue, (double)p) * inner_a;
        sum += fe * pow(r - e, (double)j) / fact * pow(ua, (double)p) * inner_e;
    }
    return sum;
}

double orc_kreg(double r, double ell, double epsB, int p)
{
    double a = 0.5 - epsB;
    double c = exp(-0.25 / (ell * ell));            /* K(1/2) */
    if (r <= a) return exp(-r * r / (ell * ell));
    if (r <= 0.5) return orc_two_point_taylor(r, a, 0.5, p, ell, c);
    return c;
}

/* ------------------------------------------------------------------------ */
/* One-axis DFT on a complex array of shape (outer, Lin, inner) producing     */
/* (outer, Lout, inner).  Input position i holds value u = i - Lin/2, output  */
/* position o holds value k = o - Lout/2;                                     */
/*   out[k] = sum_u in[u] exp(sgn 2 pi i k u / Ndft).                         */
/* Twiddles are reduced exactly as (k u mod Ndft).                            */
/* ------------------------------------------------------------------------ */
static void dft_axis(const double *in_re, const double *in_im, long outer, long Lin, long inner,
                     double *out_re, double *out_im, long Lout, long Ndft, int sgn)
{
#pragma omp parallel for schedule(static)
    for (long o0 = 0; o0 < outer; o0++) {
        for (long o = 0; o < Lout; o++) {
            long k = o - Lout / 2;
            for (long s = 0; s < inner; s++) {
                double ar = 0.0, ai = 0.0;
                for (long i = 0; i < Lin; i++) {
                    long u = i - Lin / 2;
                    long r = (k * u) % Ndft;
                    if (r < 0) r += Ndft;
                    double ang = sgn * 2.0 * M_PI * (double)r / (double)Ndft;
                    double cr = cos(ang), ci = sin(ang);
                    double xr = in_re[(o0 * Lin + i) * inner + s];
                    double xi = in_im ? in_im[(o0 * Lin + i) * inner + s] : 0.0;
                    ar += xr * cr - xi * ci;
                    ai += xr * ci + xi * cr;
                }
                out_re[(o0 * Lout + o) * inner + s] = ar;
                out_im[(o0 * Lout + o) * inner + s] = ai;
            }
        }
    }
}

/* d-dimensional transform, one axis after the other.  Input extents Lin per
 * axis, output Lout per axis, DFT length Ndft.  Arrays are row-major with the
 * last axis fastest. */
static void dft_nd(const double *in_re, const double *in_im, int dA, long Lin, long Lout, long Ndft,
                   int sgn, double *out_re, double *out_im)
{
    long maxlen = ipow(Lin > Lout ? Lin : Lout, dA);
    double *ar = calloc(maxlen, sizeof(double)), *ai = calloc(maxlen, sizeof(double));
    double *br = calloc(maxlen, sizeof(double)), *bi = calloc(maxlen, sizeof(double));
    long cur = ipow(Lin, dA);
    memcpy(ar, in_re, cur * sizeof(double));
    if (in_im) memcpy(ai, in_im, cur * sizeof(double));
    /* shape: axes 0..t-1 already Lout, axes t..dA-1 still Lin */
    for (int t = 0; t < dA; t++) {
        long outer = ipow(Lout, t);
        long inner = ipow(Lin, dA - t - 1);
        dft_axis(ar, ai, outer, Lin, inner, br, bi, Lout, Ndft, sgn);
        long nxt = outer * Lout * inner;
        memcpy(ar, br, nxt * sizeof(double));
        memcpy(ai, bi, nxt * sizeof(double));
    }
    long fin = ipow(Lout, dA);
    memcpy(out_re, ar, fin * sizeof(double));
    memcpy(out_im, ai, fin * sizeof(double));
    free(ar); free(ai); free(br); free(bi);
}

/* ------------------------------------------------------------------------ */
/* Kernel Fourier coefficients (Sec. 4.2: "ordinary FFT of M equidistant     */
/* samples of the periodic function"), here a naive DFT:                     */
/*   b_k = n^{-dA} sum_{j in I_n^dA} K_R(||j||/n) exp(-2 pi i k.j / n)        */
/* Real and imaginary parts are returned separately (the latter vanishes).   */
/* ------------------------------------------------------------------------ */
void orc_kernel_coeffs(int dA, int n, double ell, double epsB, int p, double *bk_re, double *bk_im)
{
    long tot = ipow(n, dA);
    double *f = malloc(tot * sizeof(double));
    for (long idx = 0; idx < tot; idx++) {
        long rem = idx;
        double r2 = 0.0;
        for (int t = dA - 1; t >= 0; t--) {
            long j = rem % n - n / 2;
            rem /= n;
            double v = (double)j / (double)n;
            r2 += v * v;
        }
        f[idx] = orc_kreg(sqrt(r2), ell, epsB, p);
    }
    dft_nd(f, NULL, dA, n, n, n, -1, bk_re, bk_im);
    double sc = 1.0 / (double)tot;
    for (long idx = 0; idx < tot; idx++) { bk_re[idx] *= sc; bk_im[idx] *= sc; }
    free(f);
}

/* D_k = b_k / prod_t phihat(k_t)^2  (Sec. 4.3, D = diag(c_k), with the window
 * deconvolution of the adjoint NFFT and of the NFFT folded in) */
void orc_diag(int dA, int n, int nos, int m, double b, const double *bk, double *D)
{
    long tot = ipow(n, dA);
    for (long idx = 0; idx < tot; idx++) {
        long rem = idx;
        double den = 1.0;
        for (int t = dA - 1; t >= 0; t--) {
            long k = rem % n - n / 2;
            rem /= n;
            double ph = orc_kb_phihat(k, nos, m, b);
            den *= ph * ph;
        }
        D[idx] = bk[idx] / den;
    }
}

/* ------------------------------------------------------------------------ */
/* Spreading (window step of the adjoint NFFT, Eq. adjnfft):                 */
/*   g_u = sum_j alpha_j prod_t phi(nos x_{j,t} - u_t),  u on the nos^dA grid */
/* xt holds torus coordinates, row-major N x dA.                              */
/* ------------------------------------------------------------------------ */
void orc_spread(const double *xt, long N, int dA, int nos, int m, double b,
                const double *alpha, double *g)
{
    long tot = ipow(nos, dA);
    memset(g, 0, tot * sizeof(double));
    int ntap = 2 * m + 2;
    long u0[3];
    double wts[3][64];
    for (long j = 0; j < N; j++) {
        for (int t = 0; t < dA; t++) {
            double y = (double)nos * xt[j * dA + t];
            u0[t] = (long)floor(y) - m;
            for (int a = 0; a < ntap; a++) wts[t][a] = orc_kb_phi(y - (double)(u0[t] + a), m, b);
        }
        long ntot = ipow(ntap, dA);
        for (long c = 0; c < ntot; c++) {
            long rem = c, pos = 0;
            double wprod = alpha[j];
            int tap[3];
            for (int t = dA - 1; t >= 0; t--) { tap[t] = rem % ntap; rem /= ntap; }
            for (int t = 0; t < dA; t++) {
                wprod *= wts[t][tap[t]];
                pos = pos * nos + centred_pos(u0[t] + tap[t], nos);
            }
            g[pos] += wprod;
        }
    }
}

/* Gather (window step of the NFFT, Eq. nfft): out_j = sum_u h_u prod_t phi(...) */
void orc_gather(const double *xt, long N, int dA, int nos, int m, double b,
                const double *h, double *out)
{
    int ntap = 2 * m + 2;
#pragma omp parallel for schedule(static)
    for (long j = 0; j < N; j++) {
        long u0[3];
        double wts[3][64];
        for (int t = 0; t < dA; t++) {
            double y = (double)nos * xt[j * dA + t];
            u0[t] = (long)floor(y) - m;
            for (int a = 0; a < ntap; a++) wts[t][a] = orc_kb_phi(y - (double)(u0[t] + a), m, b);
        }
        long ntot = ipow(ntap, dA);
        double acc = 0.0;
        for (long c = 0; c < ntot; c++) {
            long rem = c, pos = 0;
            double wprod = 1.0;
            int tap[3];
            for (int t = dA - 1; t >= 0; t--) { tap[t] = rem % ntap; rem /= ntap; }
            for (int t = 0; t < dA; t++) {
                wprod *= wts[t][tap[t]];
                pos = pos * nos + centred_pos(u0[t] + tap[t], nos);
            }
            acc += wprod * h[pos];
        }
        out[j] = acc;
    }
}

/* Forward transform of a real grid to the frequencies k in I_n^dA:
 *   G_k = sum_u g_u exp(-2 pi i k.u / nos) */
void orc_grid_dft(const double *g, int dA, int nos, int n, double *G_re, double *G_im)
{
    dft_nd(g, NULL, dA, nos, n, nos, -1, G_re, G_im);
}

/* Inverse transform with zero padding:  h_u = sum_{k in I_n} H_k exp(2 pi i k.u / nos) */
void orc_grid_idft(const double *H_re, const double *H_im, int dA, int nos, int n,
                   double *h_re, double *h_im)
{
    dft_nd(H_re, H_im, dA, n, nos, nos, +1, h_re, h_im);
}

/* ------------------------------------------------------------------------ */
/* O4: brute-force NDFTs on torus nodes, Eq. (adjnfft) and Eq. (nfft).       */
/* ------------------------------------------------------------------------ */
void orc_adjoint_ndft(const double *xt, long N, int dA, int n, const double *c,
                      double *g_re, double *g_im)
{
    long tot = ipow(n, dA);
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < tot; idx++) {
        long rem = idx, k[3] = {0, 0, 0};
        for (int t = dA - 1; t >= 0; t--) { k[t] = rem % n - n / 2; rem /= n; }
        double ar = 0.0, ai = 0.0;
        for (long j = 0; j < N; j++) {
            double ph = 0.0;
            for (int t = 0; t < dA; t++) ph += (double)k[t] * xt[j * dA + t];
            ar += c[j] * cos(-2.0 * M_PI * ph);
            ai += c[j] * sin(-2.0 * M_PI * ph);
        }
        g_re[idx] = ar;
        g_im[idx] = ai;
    }
}

/* adjoint NFFT with the window method: spread, DFT, divide by phihat. */
void orc_adjoint_nfft(const double *xt, long N, int dA, int n, int nos, int m, double b,
                      const double *c, double *g_re, double *g_im)
{
    long tg = ipow(nos, dA), tk = ipow(n, dA);
    double *grid = malloc(tg * sizeof(double));
    orc_spread(xt, N, dA, nos, m, b, c, grid);
    orc_grid_dft(grid, dA, nos, n, g_re, g_im);
    for (long idx = 0; idx < tk; idx++) {
        long rem = idx;
        double den = 1.0;
        for (int t = dA - 1; t >= 0; t--) { long k = rem % n - n / 2; rem /= n; den *= orc_kb_phihat(k, nos, m, b); }
        g_re[idx] /= den;
        g_im[idx] /= den;
    }
    free(grid);
}

/* NFFT with the window method, real part only (the tests use real-even data) */
void orc_nfft_real(const double *xt, long N, int dA, int n, int nos, int m, double b,
                   const double *f_re, const double *f_im, double *out)
{
    long tg = ipow(nos, dA), tk = ipow(n, dA);
    double *hr = malloc(tk * sizeof(double)), *hi = malloc(tk * sizeof(double));
    double *gr = malloc(tg * sizeof(double)), *gi = malloc(tg * sizeof(double));
    for (long idx = 0; idx < tk; idx++) {
        long rem = idx;
        double den = 1.0;
        for (int t = dA - 1; t >= 0; t--) { long k = rem % n - n / 2; rem /= n; den *= orc_kb_phihat(k, nos, m, b); }
        hr[idx] = f_re[idx] / den;
        hi[idx] = f_im[idx] / den;
    }
    orc_grid_idft(hr, hi, dA, nos, n, gr, gi);
    orc_gather(xt, N, dA, nos, m, b, gr, out);
    free(hr); free(hi); free(gr); free(gi);
}

/* ------------------------------------------------------------------------ */
/* O2: one window of the fast summation (Eq. fastsum, Sec. 4.3):             */
/*   s_i = sum_u Re(h_u) prod phi(nos z_i - u),  h = IDFT(D . DFT(g)),        */
/*   g = spread(alpha at x).  Torus coordinates are given.                    */
/* If grid_out is non-NULL it receives the spread grid g (nos^dA).            */
/* ------------------------------------------------------------------------ */
void orc_fastsum_window(const double *zt, long Nz, const double *xt, long Nx, int dA,
                        int n, int nos, int m, double b, const double *D,
                        const double *alpha, double *out, double *grid_out, double *imag_max)
{
    long tg = ipow(nos, dA), tk = ipow(n, dA);
    double *g = malloc(tg * sizeof(double));
    double *Gr = malloc(tk * sizeof(double)), *Gi = malloc(tk * sizeof(double));
    double *hr = malloc(tg * sizeof(double)), *hi = malloc(tg * sizeof(double));
    orc_spread(xt, Nx, dA, nos, m, b, alpha, g);
    if (grid_out) memcpy(grid_out, g, tg * sizeof(double));
    orc_grid_dft(g, dA, nos, n, Gr, Gi);
    for (long idx = 0; idx < tk; idx++) { Gr[idx] *= D[idx]; Gi[idx] *= D[idx]; }
    orc_grid_idft(Gr, Gi, dA, nos, n, hr, hi);
    if (imag_max) {
        double mi = 0.0, mr = 0.0;
        for (long idx = 0; idx < tg; idx++) {
            if (fabs(hi[idx]) > mi) mi = fabs(hi[idx]);
            if (fabs(hr[idx]) > mr) mr = fabs(hr[idx]);
        }
        *imag_max = (mr > 0.0) ? mi / mr : mi;
    }
    orc_gather(zt, Nz, dA, nos, m, b, hr, out);
    free(g); free(Gr); free(Gi); free(hr); free(hi);
}

/* torus coordinates of one window: xt = s (x - centre) */
static void window_coords(const double *X, long N, long ld, const int *w, const double *centre,
                          double s, double *xt)
{
    int dA = win_dim(w);
    for (long j = 0; j < N; j++)
        for (int t = 0; t < dA; t++) xt[j * dA + t] = s * (X[j * ld + w[t]] - centre[t]);
}

/* Full fast ANOVA summation, Sec. 4.3 and Sec. 5:
 *   out_i = sum_l eta_l s_l(z_i).
 * Z == X gives K alpha.  For Z != X the window frame comes from X alone when
 * every z lands inside the ball, otherwise from X and Z together.
 * nvec: bandwidth n per window; nos = sigma n.  Returns 0 on success. */
int orc_fastsum(const double *Z, long Nz, long ldz,
                const double *X, long Nx, long ldx,
                const int *win, int P, const double *eta, double ell,
                const int *nvec, int m, double sigma, double epsB, int p,
                const double *alpha, double *out)
{
    const double RB = 0.25 - 0.5 * epsB;
    const double b = M_PI * (2.0 - 1.0 / sigma);
    int same = (Z == X);
    for (long i = 0; i < Nz; i++) out[i] = 0.0;
    for (int l = 0; l < P; l++) {
        const int *w = win + 3 * l;
        int dA = win_dim(w);
        if (dA < 1) return 1;
        int n = nvec[l];
        int nos = (int)lround(sigma * n);
        double centre[3], s;
        orc_window_frame(X, Nx, ldx, NULL, 0, 0, w, RB, centre, &s);
        if (!same) {
            double rmax = 0.0;
            for (long i = 0; i < Nz; i++) {
                double r2 = 0.0;
                for (int t = 0; t < dA; t++) {
                    double df = Z[i * ldz + w[t]] - centre[t];
                    r2 += df * df;
                }
                if (r2 > rmax) rmax = r2;
            }
            if (s * sqrt(rmax) > RB) orc_window_frame(X, Nx, ldx, Z, Nz, ldz, w, RB, centre, &s);
        }
        double ell_l = s * ell;
        long tk = ipow(n, dA);
        double *bre = malloc(tk * sizeof(double)), *bim = malloc(tk * sizeof(double));
        double *D = malloc(tk * sizeof(double));
        orc_kernel_coeffs(dA, n, ell_l, epsB, p, bre, bim);
        orc_diag(dA, n, nos, m, b, bre, D);
        double *xt = malloc(Nx * dA * sizeof(double));
        window_coords(X, Nx, ldx, w, centre, s, xt);
        double *zt = xt;
        if (!same) {
            zt = malloc(Nz * dA * sizeof(double));
            window_coords(Z, Nz, ldz, w, centre, s, zt);
        }
        double *sl = malloc(Nz * sizeof(double));
        orc_fastsum_window(zt, Nz, xt, Nx, dA, n, nos, m, b, D, alpha, sl, NULL, NULL);
        for (long i = 0; i < Nz; i++) out[i] += eta[l] * sl[i];
        free(sl);
        if (!same) free(zt);
        free(xt); free(bre); free(bim); free(D);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* O3: conjugate gradients (Hestenes-Stiefel) on (K + lambda I) alpha = y,    */
/* Sec. 2.  alpha_0 = 0; stop when the recursive residual satisfies           */
/* ||r|| <= tol ||y|| or after maxit iterations.  K is the fast operator      */
/* (use_direct = 0) or the direct sum (use_direct = 1).  Returns the number of */
/* iterations; *relres receives the true residual recomputed at the end.     */
/* ------------------------------------------------------------------------ */
static void apply_op(int use_direct, const double *X, long N, long ld, const int *win, int P,
                     const double *eta, double ell, const int *nvec, int m, double sigma,
                     double epsB, int p, double lambda, const double *v, double *out)
{
    if (use_direct) orc_direct(X, N, ld, X, N, ld, win, P, eta, ell, v, out);
    else orc_fastsum(X, N, ld, X, N, ld, win, P, eta, ell, nvec, m, sigma, epsB, p, v, out);
    for (long i = 0; i < N; i++) out[i] += lambda * v[i];
}

static double dot(const double *a, const double *b, long N)
{
    double s = 0.0;
    for (long i = 0; i < N; i++) s += a[i] * b[i];
    return s;
}

int orc_cg(const double *X, long N, long ld, const int *win, int P, const double *eta, double ell,
           const int *nvec, int m, double sigma, double epsB, int p, int use_direct,
           double lambda, const double *y, double tol, int maxit, double *alpha, double *relres)
{
    double *r = malloc(N * sizeof(double)), *pv = malloc(N * sizeof(double));
    double *q = malloc(N * sizeof(double));
    for (long i = 0; i < N; i++) { alpha[i] = 0.0; r[i] = y[i]; pv[i] = y[i]; }
    double yy = dot(y, y, N), rr = yy;
    int it = 0;
    while (it < maxit && rr > tol * tol * yy) {
        apply_op(use_direct, X, N, ld, win, P, eta, ell, nvec, m, sigma, epsB, p, lambda, pv, q);
        double a = rr / dot(pv, q, N);
        for (long i = 0; i < N; i++) { alpha[i] += a * pv[i]; r[i] -= a * q[i]; }
        double rr_new = dot(r, r, N);
        double beta = rr_new / rr;
        for (long i = 0; i < N; i++) pv[i] = r[i] + beta * pv[i];
        rr = rr_new;
        it++;
    }
    apply_op(use_direct, X, N, ld, win, P, eta, ell, nvec, m, sigma, epsB, p, lambda, alpha, q);
    for (long i = 0; i < N; i++) r[i] = y[i] - q[i];
    *relres = sqrt(dot(r, r, N) / yy);
    free(r); free(pv); free(q);
    return it;
}
