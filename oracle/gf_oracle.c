/*
 * Plain FP64 CPU oracle for the lattice Green's function path of
 * "Implementation of LDA+DMFT with pseudo-potential-plane-wave method"
 * (Zhao et al., arXiv:1111.2157).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA library
 * shares no code, header, table or helper with it.
 *
 * Everything here is the definition written out, in complex double precision,
 * one (k, i w_n) point at a time:
 *
 *   w_n    = (2n+1) pi / beta, n = 0..N_w-1          (fermionic Matsubara grid)
 *   A      = (i w_n + mu) I - H_k - P_k^+ Sigma(i w_n) P_k      (Sec. 3.2.2, Eq. dmftloop1)
 *   G      = A^{-1}   (LU with partial pivoting, then N_b solves)
 *   G_loc  = sum_k w_k P_k G P_k^+                    (Sec. 3.2.2, the k-sum inside Eq. dmftloop2)
 *   rho_k  = (1/beta) sum_{n in Z} G(i w_n) e^{i w_n 0+}   (Sec. 3.3, Eq. rho_LDA+DMFT)
 *          = (1/beta) sum_{n=0}^{N_w-1} [(G-T) + (G-T)^+] + I/2 - (beta/4) M2
 *            with T = I/(i w_n) + M2/(i w_n)^2 and M2 = H_k + P_k^+ Sigma(inf) P_k - mu I
 *   N      = sum_k w_k Tr rho_k                       (Sec. 3.3, Eq. fix_mu)
 *   n_corr = sum_k w_k Tr(P_k rho_k P_k^+)            (Sec. 3.4, Eq. nf_LDA+DMFT)
 *   dN/dmu = sum_k w_k Tr d rho_k/d mu, d rho_k/d mu = (1/beta) sum_n [(-G^2 + I/(i w_n)^2) + h.c.] + (beta/4) I
 *
 * The tail T, the use of G(-i w_n) = G(i w_n)^+ for the negative frequencies,
 * and the exact sums (1/beta) sum_{n in Z} e^{i w_n 0+}/(i w_n) = 1/2 and
 * (1/beta) sum_{n in Z} 1/(i w_n)^2 = -beta/4 are this implementation's reading:
 * the paper writes the frequency sum of Eq. rho_LDA+DMFT without a tail.
 * With tail_order = 1 the M2 terms are dropped.
 *
 * Adjoint (not in the paper; derived from the definitions above, with
 * dG = G (P^+ dSigma P) G and dG/dmu = -G^2), for a real loss L and the
 * convention grad z = dL/dRe z + i dL/dIm z:
 *   A_k = P_k G P_k^+, B_k = P_k G G P_k^+
 *   Sigma_bar(w_n) = sum_k w_k [ A_k^+ Gloc_bar(w_n) A_k^+ + N_bar (2/beta) B_k^+ ]
 *   mu_bar         = N_bar dN/dmu - sum_n sum_k w_k Re < Gloc_bar(w_n), B_k >
 *
 * Layouts (row-major, complex numbers as interleaved (re, im) doubles):
 *   H   : per k an nb[k] x nb[k] block, blocks packed back to back
 *   P   : per k an m x nb[k] block (P[a][n] = <alpha_k | phi_nk>), packed
 *   sig : [n_w][m][m];  sig_inf : [m][m];  gloc : [n_w][m][m]
 *   rho : per k an nb[k] x nb[k] block, packed like H
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static int g_threads = 0;

void gfo_set_threads(int n) { g_threads = n; }

int gfo_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

double gfo_matsubara(int n, double beta) { return (2.0 * n + 1.0) * M_PI / beta; }

/* ---------------------------------------------------------------- linear algebra */

/* In-place LU factorisation with partial pivoting (largest modulus in the
 * column, first index on ties).  Returns -1 if a pivot is exactly zero. */
static int lu_factor(int n, cplx *a, int *piv)
{
    for (int j = 0; j < n; j++) {
        int p = j;
        double best = cabs(a[j * n + j]);
        for (int i = j + 1; i < n; i++) {
            double v = cabs(a[i * n + j]);
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0) return -1;
        piv[j] = p;
        if (p != j) {
            for (int c = 0; c < n; c++) {
                cplx t = a[j * n + c]; a[j * n + c] = a[p * n + c]; a[p * n + c] = t;
            }
        }
        cplx inv = 1.0 / a[j * n + j];
        for (int i = j + 1; i < n; i++) {
            cplx l = a[i * n + j] * inv;
            a[i * n + j] = l;
            for (int c = j + 1; c < n; c++) a[i * n + c] -= l * a[j * n + c];
        }
    }
    return 0;
}

/* X = A^{-1} from the LU factors: solve A x = e_c for every column c. */
static void lu_inverse(int n, const cplx *lu, const int *piv, cplx *x, cplx *col)
{
    for (int c = 0; c < n; c++) {
        for (int i = 0; i < n; i++) col[i] = (i == c) ? 1.0 : 0.0;
        for (int j = 0; j < n; j++) {
            if (piv[j] != j) { cplx t = col[j]; col[j] = col[piv[j]]; col[piv[j]] = t; }
        }
        for (int i = 0; i < n; i++)
            for (int j = 0; j < i; j++) col[i] -= lu[i * n + j] * col[j];
        for (int i = n - 1; i >= 0; i--) {
            for (int j = i + 1; j < n; j++) col[i] -= lu[i * n + j] * col[j];
            col[i] /= lu[i * n + i];
        }
        for (int i = 0; i < n; i++) x[i * n + c] = col[i];
    }
}

/* E = P^+ S P  (nb x nb), with P m x nb and S m x m; T is m x nb scratch. */
static void embed(int nb, int m, const cplx *P, const cplx *S, cplx *E, cplx *T)
{
    for (int a = 0; a < m; a++)
        for (int j = 0; j < nb; j++) {
            cplx s = 0;
            for (int b = 0; b < m; b++) s += S[a * m + b] * P[b * nb + j];
            T[a * nb + j] = s;
        }
    for (int i = 0; i < nb; i++)
        for (int j = 0; j < nb; j++) {
            cplx s = 0;
            for (int a = 0; a < m; a++) s += conj(P[a * nb + i]) * T[a * nb + j];
            E[i * nb + j] = s;
        }
}

/* Q = P X P^+  (m x m) for an nb x nb matrix X; Y is nb x m scratch. */
static void project(int nb, int m, const cplx *P, const cplx *X, cplx *Q, cplx *Y)
{
    for (int i = 0; i < nb; i++)
        for (int b = 0; b < m; b++) {
            cplx s = 0;
            for (int j = 0; j < nb; j++) s += X[i * nb + j] * conj(P[b * nb + j]);
            Y[i * m + b] = s;
        }
    for (int a = 0; a < m; a++)
        for (int b = 0; b < m; b++) {
            cplx s = 0;
            for (int i = 0; i < nb; i++) s += P[a * nb + i] * Y[i * m + b];
            Q[a * m + b] = s;
        }
}

/* --------------------------------------------------------------- per-k workspace */

typedef struct {
    cplx *A, *G, *E, *T, *Y, *col, *G2;
    int *piv;
} work_t;

static int work_alloc(work_t *w, int nb, int m)
{
    size_t n2 = (size_t)nb * nb;
    w->A = malloc(sizeof(cplx) * n2);
    w->G = malloc(sizeof(cplx) * n2);
    w->E = malloc(sizeof(cplx) * n2);
    w->G2 = malloc(sizeof(cplx) * n2);
    w->T = malloc(sizeof(cplx) * (size_t)m * nb + 1);
    w->Y = malloc(sizeof(cplx) * (size_t)m * nb + 1);
    w->col = malloc(sizeof(cplx) * nb);
    w->piv = malloc(sizeof(int) * nb);
    return (w->A && w->G && w->E && w->G2 && w->T && w->Y && w->col && w->piv) ? 0 : -1;
}

static void work_free(work_t *w)
{
    free(w->A); free(w->G); free(w->E); free(w->G2); free(w->T); free(w->Y); free(w->col); free(w->piv);
}

/* G = [(i wn + mu) I - H - P^+ S P]^{-1} (Eq. dmftloop1).  Returns -1 if singular. */
static int green_point(int nb, int m, const cplx *H, const cplx *P, const cplx *S,
                       double wn, double mu, work_t *w)
{
    embed(nb, m, P, S, w->E, w->T);
    for (int i = 0; i < nb; i++)
        for (int j = 0; j < nb; j++)
            w->A[i * nb + j] = ((i == j) ? (mu + I * wn) : 0.0) - H[i * nb + j] - w->E[i * nb + j];
    if (lu_factor(nb, w->A, w->piv)) return -1;
    lu_inverse(nb, w->A, w->piv, w->G, w->col);
    return 0;
}

static void offsets(int nk, const int *nb, int m, size_t *offH, size_t *offP, int *nbmax)
{
    size_t h = 0, p = 0;
    int mx = 0;
    for (int k = 0; k < nk; k++) {
        offH[k] = h; offP[k] = p;
        h += (size_t)nb[k] * nb[k];
        p += (size_t)m * nb[k];
        if (nb[k] > mx) mx = nb[k];
    }
    *nbmax = mx;
}

/* ------------------------------------------------------------------ entry points */

/* One lattice Green's function G(k, i w_n), nb x nb. */
int gfo_green(int nb, int m, const double *H, const double *P, const double *sig,
              double wn, double mu, double *G)
{
    work_t w;
    if (work_alloc(&w, nb, m)) { work_free(&w); return -2; }
    int rc = green_point(nb, m, (const cplx *)H, (const cplx *)P, (const cplx *)sig, wn, mu, &w);
    if (rc == 0) memcpy(G, w.G, sizeof(cplx) * (size_t)nb * nb);
    work_free(&w);
    return rc;
}

/* G_loc(i w_n) = sum_k w_k P_k G P_k^+ at the listed frequency indices n_idx[f]
 * (sig holds Sigma at those frequencies, [n_freq][m][m]). */
int gfo_local(int nk, const int *nb, int m, const double *H_, const double *P_, const double *wk,
              int n_freq, const int *n_idx, const double *sig_, double beta, double mu, double *gloc_)
{
    const cplx *H = (const cplx *)H_, *P = (const cplx *)P_, *sig = (const cplx *)sig_;
    cplx *gloc = (cplx *)gloc_;
    size_t *offH = malloc(sizeof(size_t) * (nk + 1)), *offP = malloc(sizeof(size_t) * (nk + 1));
    int nbmax;
    offsets(nk, nb, m, offH, offP, &nbmax);
    size_t mm = (size_t)m * m;
    memset(gloc, 0, sizeof(cplx) * mm * n_freq);
    int nthr = gfo_get_threads();
    cplx *part = calloc((size_t)nthr * mm * n_freq, sizeof(cplx));
    int err = 0;
#pragma omp parallel num_threads(nthr)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        work_t w;
        cplx *Q = malloc(sizeof(cplx) * mm);
        if (work_alloc(&w, nbmax, m) || !Q) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (int k = 0; k < nk; k++) {
                for (int f = 0; f < n_freq; f++) {
                    double wn = gfo_matsubara(n_idx[f], beta);
                    if (green_point(nb[k], m, H + offH[k], P + offP[k], sig + f * mm, wn, mu, &w)) {
#pragma omp atomic write
                        err = -1;
                        continue;
                    }
                    project(nb[k], m, P + offP[k], w.G, Q, w.Y);
                    cplx *acc = part + ((size_t)t * n_freq + f) * mm;
                    for (size_t q = 0; q < mm; q++) acc[q] += wk[k] * Q[q];
                }
            }
        }
        work_free(&w);
        free(Q);
    }
    for (int t = 0; t < nthr; t++)
        for (size_t q = 0; q < mm * n_freq; q++) gloc[q] += part[(size_t)t * mm * n_freq + q];
    free(part); free(offH); free(offP);
    return err;
}

/* Full Matsubara sum: rho_k (optional), and out3 = {N, n_corr, dN/dmu}. */
int gfo_density(int nk, const int *nb, int m, const double *H_, const double *P_, const double *wk,
                int n_iw, const double *sig_, const double *sig_inf_, double beta, double mu,
                int tail_order, double *rho_, double *out3)
{
    const cplx *H = (const cplx *)H_, *P = (const cplx *)P_, *sig = (const cplx *)sig_;
    const cplx *sig_inf = (const cplx *)sig_inf_;
    cplx *rho = (cplx *)rho_;
    size_t *offH = malloc(sizeof(size_t) * (nk + 1)), *offP = malloc(sizeof(size_t) * (nk + 1));
    int nbmax;
    offsets(nk, nb, m, offH, offP, &nbmax);
    size_t mm = (size_t)m * m;
    int nthr = gfo_get_threads();
    double *partN = calloc((size_t)nthr * 3, sizeof(double));
    int err = 0;
#pragma omp parallel num_threads(nthr)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        work_t w;
        cplx *acc = malloc(sizeof(cplx) * (size_t)nbmax * nbmax);
        cplx *M2 = malloc(sizeof(cplx) * (size_t)nbmax * nbmax);
        cplx *rk = malloc(sizeof(cplx) * (size_t)nbmax * nbmax);
        cplx *Q = malloc(sizeof(cplx) * mm);
        if (work_alloc(&w, nbmax, m) || !acc || !M2 || !rk || !Q) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (int k = 0; k < nk; k++) {
                int n = nb[k];
                const cplx *Hk = H + offH[k], *Pk = P + offP[k];
                /* M2 = H_k + P^+ Sigma(inf) P - mu I : the 1/(i w)^2 moment of G. */
                embed(n, m, Pk, sig_inf, w.E, w.T);
                for (int i = 0; i < n; i++)
                    for (int j = 0; j < n; j++)
                        M2[i * n + j] = Hk[i * n + j] + w.E[i * n + j] - ((i == j) ? mu : 0.0);
                memset(acc, 0, sizeof(cplx) * n * n);
                double trG2 = 0.0; /* sum_n Re Tr(-G^2 - I/w_n^2) */
                for (int f = 0; f < n_iw; f++) {
                    double wn = gfo_matsubara(f, beta);
                    if (green_point(n, m, Hk, Pk, sig + f * mm, wn, mu, &w)) {
#pragma omp atomic write
                        err = -1;
                        continue;
                    }
                    cplx iw = I * wn;
                    for (int i = 0; i < n; i++)
                        for (int j = 0; j < n; j++) {
                            cplx tail = ((i == j) ? 1.0 / iw : 0.0);
                            if (tail_order >= 2) tail += M2[i * n + j] / (iw * iw);
                            acc[i * n + j] += w.G[i * n + j] - tail;
                        }
                    cplx tr = 0;
                    for (int i = 0; i < n; i++)
                        for (int j = 0; j < n; j++) tr += w.G[i * n + j] * w.G[j * n + i];
                    trG2 += creal(-tr);
                    if (tail_order >= 2) trG2 += -(double)n / (wn * wn);
                }
                /* rho_k = (1/beta)(acc + acc^+) + I/2 - (beta/4) M2 */
                for (int i = 0; i < n; i++)
                    for (int j = 0; j < n; j++) {
                        cplx v = (acc[i * n + j] + conj(acc[j * n + i])) / beta;
                        if (i == j) v += 0.5;
                        if (tail_order >= 2) v -= 0.25 * beta * M2[i * n + j];
                        rk[i * n + j] = v;
                    }
                if (rho) memcpy(rho + offH[k], rk, sizeof(cplx) * n * n);
                double tr = 0.0;
                for (int i = 0; i < n; i++) tr += creal(rk[i * n + i]);
                project(n, m, Pk, rk, Q, w.Y);
                double trc = 0.0;
                for (int a = 0; a < m; a++) trc += creal(Q[a * m + a]);
                double dn = 2.0 / beta * trG2;
                if (tail_order >= 2) dn += 0.25 * beta * n;
                partN[3 * t + 0] += wk[k] * tr;
                partN[3 * t + 1] += wk[k] * trc;
                partN[3 * t + 2] += wk[k] * dn;
            }
        }
        work_free(&w);
        free(acc); free(M2); free(rk); free(Q);
    }
    out3[0] = out3[1] = out3[2] = 0.0;
    for (int t = 0; t < nthr; t++)
        for (int q = 0; q < 3; q++) out3[q] += partN[3 * t + q];
    free(partN); free(offH); free(offP);
    return err;
}

/* Chemical potential: N(mu) = n_target (Sec. 3.3, Eq. fix_mu).  N is strictly
 * increasing in mu.  The bracket [mu_lo, mu_hi] is widened until it encloses
 * the root, then Brent's method (inverse quadratic interpolation / secant with
 * a bisection safeguard, R. P. Brent 1973) runs until |N - n_target| <= tol. */
int gfo_find_mu(int nk, const int *nb, int m, const double *H, const double *P, const double *wk,
                int n_iw, const double *sig, const double *sig_inf, double beta, int tail_order,
                double n_target, double mu_lo, double mu_hi, double tol, int max_iter,
                double *mu_out, double *n_out, int *iters_out)
{
    double o[3];
    int it = 0;
    double a = mu_lo, b = mu_hi, fa, fb;
    if (gfo_density(nk, nb, m, H, P, wk, n_iw, sig, sig_inf, beta, a, tail_order, NULL, o)) return -1;
    fa = o[0] - n_target; it++;
    if (gfo_density(nk, nb, m, H, P, wk, n_iw, sig, sig_inf, beta, b, tail_order, NULL, o)) return -1;
    fb = o[0] - n_target; it++;
    while (fa > 0 && it < max_iter) {
        double width = b - a; b = a; fb = fa; a -= 2 * width;
        if (gfo_density(nk, nb, m, H, P, wk, n_iw, sig, sig_inf, beta, a, tail_order, NULL, o)) return -1;
        fa = o[0] - n_target; it++;
    }
    while (fb < 0 && it < max_iter) {
        double width = b - a; a = b; fa = fb; b += 2 * width;
        if (gfo_density(nk, nb, m, H, P, wk, n_iw, sig, sig_inf, beta, b, tail_order, NULL, o)) return -1;
        fb = o[0] - n_target; it++;
    }
    if (fa > 0 || fb < 0) return -3;
    /* Brent: b is the best iterate, a the previous one, c the contrapoint. */
    double c = a, fc = fa, d = b - a, e = d;
    while (it < max_iter) {
        if ((fb > 0 && fc > 0) || (fb < 0 && fc < 0)) { c = a; fc = fa; d = e = b - a; }
        if (fabs(fc) < fabs(fb)) { a = b; b = c; c = a; fa = fb; fb = fc; fc = fa; }
        if (fabs(fb) <= tol) break;
        double xm = 0.5 * (c - b);
        double tol1 = 4e-16 * fabs(b) + 1e-15;
        if (fabs(xm) <= tol1) break;
        if (fabs(e) >= tol1 && fabs(fa) > fabs(fb)) {
            double s = fb / fa, p, q;
            if (a == c) {
                p = 2.0 * xm * s; q = 1.0 - s;
            } else {
                double qq = fa / fc, r = fb / fc;
                p = s * (2.0 * xm * qq * (qq - r) - (b - a) * (r - 1.0));
                q = (qq - 1.0) * (r - 1.0) * (s - 1.0);
            }
            if (p > 0) q = -q; else p = -p;
            if (2.0 * p < fmin(3.0 * xm * q - fabs(tol1 * q), fabs(e * q))) { e = d; d = p / q; }
            else { d = xm; e = d; }
        } else { d = xm; e = d; }
        a = b; fa = fb;
        b += (fabs(d) > tol1) ? d : (xm > 0 ? tol1 : -tol1);
        if (gfo_density(nk, nb, m, H, P, wk, n_iw, sig, sig_inf, beta, b, tail_order, NULL, o)) return -1;
        fb = o[0] - n_target; it++;
    }
    *mu_out = b;
    *n_out = fb + n_target;
    *iters_out = it;
    return fabs(fb) <= tol ? 0 : -4;
}

/* Vector-Jacobian product of (G_loc, N) with respect to (Sigma(i w_n), mu). */
int gfo_backward(int nk, const int *nb, int m, const double *H_, const double *P_, const double *wk,
                 int n_iw, const double *sig_, const double *sig_inf_, double beta, double mu,
                 int tail_order, const double *gbar_, double n_bar, double *sbar_, double *mu_bar)
{
    const cplx *H = (const cplx *)H_, *P = (const cplx *)P_, *sig = (const cplx *)sig_;
    const cplx *gbar = (const cplx *)gbar_;
    cplx *sbar = (cplx *)sbar_;
    size_t *offH = malloc(sizeof(size_t) * (nk + 1)), *offP = malloc(sizeof(size_t) * (nk + 1));
    int nbmax;
    offsets(nk, nb, m, offH, offP, &nbmax);
    size_t mm = (size_t)m * m;
    int nthr = gfo_get_threads();
    cplx *part = calloc((size_t)nthr * mm * n_iw, sizeof(cplx));
    double *pmu = calloc((size_t)nthr, sizeof(double));
    int err = 0;
    double o[3];
    if (n_bar != 0.0) {
        if (gfo_density(nk, nb, m, H_, P_, wk, n_iw, sig_, sig_inf_, beta, mu, tail_order, NULL, o)) err = -1;
    } else {
        o[2] = 0.0;
    }
#pragma omp parallel num_threads(nthr)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        work_t w;
        cplx *Ak = malloc(sizeof(cplx) * mm), *Bk = malloc(sizeof(cplx) * mm);
        cplx *Z = malloc(sizeof(cplx) * (size_t)m * nbmax), *Mt = malloc(sizeof(cplx) * mm);
        if (work_alloc(&w, nbmax, m) || !Ak || !Bk || !Z || !Mt) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (int k = 0; k < nk; k++) {
                int n = nb[k];
                const cplx *Hk = H + offH[k], *Pk = P + offP[k];
                for (int f = 0; f < n_iw; f++) {
                    double wn = gfo_matsubara(f, beta);
                    if (green_point(n, m, Hk, Pk, sig + f * mm, wn, mu, &w)) {
#pragma omp atomic write
                        err = -1;
                        continue;
                    }
                    /* Y = G P^+ (n x m), A_k = P Y, Z = P G (m x n), B_k = Z Y */
                    project(n, m, Pk, w.G, Ak, w.Y);
                    for (int a = 0; a < m; a++)
                        for (int j = 0; j < n; j++) {
                            cplx s = 0;
                            for (int i = 0; i < n; i++) s += Pk[a * n + i] * w.G[i * n + j];
                            Z[a * n + j] = s;
                        }
                    for (int a = 0; a < m; a++)
                        for (int b = 0; b < m; b++) {
                            cplx s = 0;
                            for (int j = 0; j < n; j++) s += Z[a * n + j] * w.Y[j * m + b];
                            Bk[a * m + b] = s;
                        }
                    cplx *acc = part + ((size_t)t * n_iw + f) * mm;
                    if (gbar) {
                        const cplx *Gb = gbar + f * mm;
                        /* Mt = Gb A^+ ; acc += w_k A^+ Mt */
                        for (int a = 0; a < m; a++)
                            for (int b = 0; b < m; b++) {
                                cplx s = 0;
                                for (int c = 0; c < m; c++) s += Gb[a * m + c] * conj(Ak[b * m + c]);
                                Mt[a * m + b] = s;
                            }
                        for (int a = 0; a < m; a++)
                            for (int b = 0; b < m; b++) {
                                cplx s = 0;
                                for (int c = 0; c < m; c++) s += conj(Ak[c * m + a]) * Mt[c * m + b];
                                acc[a * m + b] += wk[k] * s;
                            }
                        double re = 0.0;
                        for (size_t q = 0; q < mm; q++) re += creal(conj(Gb[q]) * Bk[q]);
                        pmu[t] -= wk[k] * re;
                    }
                    if (n_bar != 0.0)
                        for (int a = 0; a < m; a++)
                            for (int b = 0; b < m; b++)
                                acc[a * m + b] += wk[k] * n_bar * (2.0 / beta) * conj(Bk[b * m + a]);
                }
            }
        }
        work_free(&w);
        free(Ak); free(Bk); free(Z); free(Mt);
    }
    memset(sbar, 0, sizeof(cplx) * mm * n_iw);
    double mb = n_bar * o[2];
    for (int t = 0; t < nthr; t++) {
        for (size_t q = 0; q < mm * n_iw; q++) sbar[q] += part[(size_t)t * mm * n_iw + q];
        mb += pmu[t];
    }
    *mu_bar = mb;
    free(part); free(pmu); free(offH); free(offP);
    return err;
}
