/*
 * Drives every routine of the FP64 oracle (oracle/anova_oracle.c) once on small
 * inputs, for a build with AddressSanitizer and UndefinedBehaviorSanitizer: an
 * out-of-bounds access, a use of uninitialised heap or an undefined operation
 * anywhere in the oracle makes the run fail.  The results are checked only for
 * finiteness here; their values are pinned by tests/test_oracle.py.
 * Test infrastructure: compiled and run by tests/test_oracle_sanitizers.py.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

void orc_direct(const double *Z, long Nz, long ldz, const double *X, long Nx, long ldx, const int *win, int P,
                const double *eta, double ell, const double *alpha, double *out);
void orc_window_frame(const double *X, long Nx, long ldx, const double *Z, long Nz, long ldz, const int *w,
                      double RB, double *centre, double *scale);
double orc_bessel_i0(double x);
double orc_kb_phi(double t, int m, double b);
double orc_kb_phihat(long k, long nos, int m, double b);
double orc_gauss_deriv(int j, double r, double ell);
double orc_two_point_taylor(double r, double a, double e, int p, double ell, double c);
double orc_kreg(double r, double ell, double epsB, int p);
void orc_kernel_coeffs(int dA, int n, double ell, double epsB, int p, double *bk_re, double *bk_im);
void orc_diag(int dA, int n, int nos, int m, double b, const double *bk, double *D);
void orc_spread(const double *xt, long N, int dA, int nos, int m, double b, const double *alpha, double *g);
void orc_gather(const double *xt, long N, int dA, int nos, int m, double b, const double *h, double *out);
void orc_grid_dft(const double *g, int dA, int nos, int n, double *G_re, double *G_im);
void orc_grid_idft(const double *H_re, const double *H_im, int dA, int nos, int n, double *h_re, double *h_im);
void orc_adjoint_ndft(const double *xt, long N, int dA, int n, const double *c, double *g_re, double *g_im);
void orc_adjoint_nfft(const double *xt, long N, int dA, int n, int nos, int m, double b, const double *c,
                      double *g_re, double *g_im);
void orc_nfft_real(const double *xt, long N, int dA, int n, int nos, int m, double b, const double *f_re,
                   const double *f_im, double *out);
void orc_fastsum_window(const double *zt, long Nz, const double *xt, long Nx, int dA, int n, int nos, int m,
                        double b, const double *D, const double *alpha, double *out, double *grid_out,
                        double *imag_max);
int orc_fastsum(const double *Z, long Nz, long ldz, const double *X, long Nx, long ldx, const int *win, int P,
                const double *eta, double ell, const int *nvec, int m, double sigma, double epsB, int p,
                const double *alpha, double *out);
int orc_cg(const double *X, long N, long ld, const int *win, int P, const double *eta, double ell, const int *nvec,
           int m, double sigma, double epsB, int p, int use_direct, double lambda, const double *y, double tol,
           int maxit, double *alpha, double *relres);

static int bad = 0;

static void check_finite(const char *what, const double *v, long n)
{
    for (long i = 0; i < n; i++)
        if (!isfinite(v[i])) {
            fprintf(stderr, "%s: entry %ld not finite\n", what, i);
            bad = 1;
            return;
        }
}

static double *vec(long n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static double urand(unsigned *s)
{
    *s = *s * 1664525u + 1013904223u;
    return (double)(*s >> 8) / 16777216.0;
}

int main(void)
{
    unsigned seed = 12345u;
    const long N = 120, d = 5;
    const double b = M_PI * 1.5;
    double *X = vec(N * d), *alpha = vec(N), *out = vec(N), *y = vec(N);
    for (long i = 0; i < N * d; i++) X[i] = urand(&seed) - 0.5;
    for (long i = 0; i < N; i++) { alpha[i] = urand(&seed) - 0.5; y[i] = urand(&seed); }
    const int win[9] = {0, 1, 2, 3, 4, -1, 2, -1, -1};
    const double eta[3] = {0.5, 0.3, 0.2};
    const int nvec[3] = {8, 16, 16};

    orc_direct(X, N, d, X, N, d, win, 3, eta, 0.2, alpha, out);
    check_finite("direct", out, N);

    double c[3], s;
    orc_window_frame(X, N, d, X, 7, d, win, 0.21875, c, &s);
    check_finite("frame", c, 3);

    double sc[6] = {orc_bessel_i0(3.0), orc_kb_phi(0.5, 4, b), orc_kb_phi(4.0, 4, b),
                    orc_kb_phihat(3, 32, 4, b), orc_gauss_deriv(7, 0.3, 0.2),
                    orc_two_point_taylor(0.45, 0.4375, 0.5, 8, 0.2, exp(-6.25))};
    check_finite("scalars", sc, 6);
    double kr = orc_kreg(0.6, 0.2, 1.0 / 16, 8);
    check_finite("kreg", &kr, 1);

    for (int dA = 1; dA <= 3; dA++) {
        const int n = dA == 3 ? 8 : 16, nos = 2 * n, m = 3;
        long tk = 1, tg = 1;
        for (int t = 0; t < dA; t++) { tk *= n; tg *= nos; }
        double *bre = vec(tk), *bim = vec(tk), *D = vec(tk), *g = vec(tg), *gi = vec(tg);
        double *Gr = vec(tk), *Gi = vec(tk), *xt = vec(N * dA), *o = vec(N);
        for (long i = 0; i < N * dA; i++) xt[i] = 0.4 * (urand(&seed) - 0.5);
        orc_kernel_coeffs(dA, n, 0.2, 1.0 / 8, 6, bre, bim);
        orc_diag(dA, n, nos, m, b, bre, D);
        orc_spread(xt, N, dA, nos, m, b, alpha, g);
        orc_gather(xt, N, dA, nos, m, b, g, o);
        orc_grid_dft(g, dA, nos, n, Gr, Gi);
        orc_grid_idft(Gr, Gi, dA, nos, n, g, gi);
        orc_adjoint_ndft(xt, N, dA, n, alpha, Gr, Gi);
        orc_adjoint_nfft(xt, N, dA, n, nos, m, b, alpha, Gr, Gi);
        orc_nfft_real(xt, N, dA, n, nos, m, b, bre, bim, o);
        double im = 0.0;
        orc_fastsum_window(xt, 17, xt, N, dA, n, nos, m, b, D, alpha, o, g, &im);
        check_finite("coeffs", bre, tk);
        check_finite("diag", D, tk);
        check_finite("grid", g, tg);
        check_finite("window", o, 17);
        free(bre); free(bim); free(D); free(g); free(gi); free(Gr); free(Gi); free(xt); free(o);
    }

    double *Z = vec(9 * d), *oz = vec(9);
    for (long i = 0; i < 9 * d; i++) Z[i] = 3.0 * (urand(&seed) - 0.5);   /* outside the ball: joint frame */
    if (orc_fastsum(X, N, d, X, N, d, win, 3, eta, 0.2, nvec, 3, 2.0, 1.0 / 8, 6, alpha, out)) bad = 1;
    if (orc_fastsum(Z, 9, d, X, N, d, win, 3, eta, 0.2, nvec, 3, 2.0, 1.0 / 8, 6, alpha, oz)) bad = 1;
    check_finite("fastsum", out, N);
    check_finite("predict", oz, 9);

    double rel = 0.0;
    orc_cg(X, N, d, win, 3, eta, 0.2, nvec, 3, 2.0, 1.0 / 8, 6, 0, 1e-2, y, 1e-8, 300, out, &rel);
    orc_cg(X, N, d, win, 3, eta, 0.2, nvec, 3, 2.0, 1.0 / 8, 6, 1, 1e-2, y, 1e-8, 300, out, &rel);
    check_finite("cg", out, N);
    check_finite("relres", &rel, 1);

    free(X); free(alpha); free(out); free(y); free(Z); free(oz);
    if (!bad) printf("oracle sanitizer run ok\n");
    return bad;
}
