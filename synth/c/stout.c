/* Stout-style smoothing of an SU(3) gauge field, for generating inputs only.
 *
 * One step, all links at once, with isotropic weight rho:
 *   C_mu(x) = rho sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
 *                                 + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
 *   Om = C_mu(x) U_mu(x)^dag,  A = Om^dag - Om,
 *   Q  = (i/2) A - (i/6) tr(A) 1            (Hermitian, traceless)
 *   U_mu(x) <- exp(i Q) U_mu(x)
 * the same recipe as stout_smooth in gauge.py; here exp(iQ) is a Taylor
 * series after scaling by 2^-s, squared back s times (scaling and squaring),
 * instead of an eigen-decomposition.
 *
 * Links: double[V][4][3][3][2] (re, im), site s = x + nx (y + ny (z + nz t)).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double re, im;
} cx;

static inline cx cmul(cx a, cx b) { cx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static inline cx cadd(cx a, cx b) { cx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cx conjx(cx a) { cx r = {a.re, -a.im}; return r; }

/* C = A B, C = A B^dag, C = A^dag B (3x3, row-major) */
static void mm(const cx *a, const cx *b, cx *c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cx s = {0, 0};
            for (int k = 0; k < 3; ++k) s = cadd(s, cmul(a[i * 3 + k], b[k * 3 + j]));
            c[i * 3 + j] = s;
        }
}
static void mmd(const cx *a, const cx *b, cx *c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cx s = {0, 0};
            for (int k = 0; k < 3; ++k) s = cadd(s, cmul(a[i * 3 + k], conjx(b[j * 3 + k])));
            c[i * 3 + j] = s;
        }
}
static void mdm(const cx *a, const cx *b, cx *c) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cx s = {0, 0};
            for (int k = 0; k < 3; ++k) s = cadd(s, cmul(conjx(a[k * 3 + i]), b[k * 3 + j]));
            c[i * 3 + j] = s;
        }
}

static int neighbour(const int *n, int s, int mu, int step) {
    int c[4] = {s % n[0], (s / n[0]) % n[1], (s / (n[0] * n[1])) % n[2], s / (n[0] * n[1] * n[2])};
    c[mu] = (c[mu] + step + n[mu]) % n[mu];
    return c[0] + n[0] * (c[1] + n[1] * (c[2] + n[2] * c[3]));
}

/* E = exp(X) for X = i Q anti-Hermitian: scaling and squaring with a
 * 14-term Taylor series */
static void expm3(const cx *x, cx *e) {
    double nrm = 0;
    for (int i = 0; i < 9; ++i) nrm += x[i].re * x[i].re + x[i].im * x[i].im;
    nrm = sqrt(nrm);
    int s = 0;
    while (nrm > 0.25) {
        nrm *= 0.5;
        ++s;
    }
    const double f = ldexp(1.0, -s);
    cx y[9], term[9], tmp[9];
    for (int i = 0; i < 9; ++i) {
        y[i].re = x[i].re * f;
        y[i].im = x[i].im * f;
        e[i].re = (i % 4 == 0) ? 1.0 : 0.0;
        e[i].im = 0.0;
        term[i] = e[i];
    }
    for (int k = 1; k <= 14; ++k) {
        mm(term, y, tmp);
        for (int i = 0; i < 9; ++i) {
            term[i].re = tmp[i].re / k;
            term[i].im = tmp[i].im / k;
            e[i] = cadd(e[i], term[i]);
        }
    }
    for (int k = 0; k < s; ++k) {
        mm(e, e, tmp);
        memcpy(e, tmp, sizeof(tmp));
    }
}

void synth_stout(double *links, const int *dims, double rho, int steps) {
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    cx *U = (cx *)links;
    cx *W = (cx *)malloc(sizeof(cx) * 36 * V);
    if (!W) return;
    for (int step = 0; step < steps; ++step) {
#pragma omp parallel for schedule(static)
        for (long s = 0; s < V; ++s) {
            for (int mu = 0; mu < 4; ++mu) {
                cx C[9], t1[9], t2[9];
                memset(C, 0, sizeof(C));
                for (int nu = 0; nu < 4; ++nu) {
                    if (nu == mu) continue;
                    const int spn = neighbour(dims, (int)s, nu, +1), spm = neighbour(dims, (int)s, mu, +1);
                    const int smn = neighbour(dims, (int)s, nu, -1), smnpm = neighbour(dims, smn, mu, +1);
                    mm(U + (s * 4 + nu) * 9, U + ((long)spn * 4 + mu) * 9, t1);
                    mmd(t1, U + ((long)spm * 4 + nu) * 9, t2);
                    for (int i = 0; i < 9; ++i) C[i] = cadd(C[i], t2[i]);
                    mdm(U + ((long)smn * 4 + nu) * 9, U + ((long)smn * 4 + mu) * 9, t1);
                    mm(t1, U + ((long)smnpm * 4 + nu) * 9, t2);
                    for (int i = 0; i < 9; ++i) C[i] = cadd(C[i], t2[i]);
                }
                for (int i = 0; i < 9; ++i) {
                    C[i].re *= rho;
                    C[i].im *= rho;
                }
                cx Om[9], A[9], X[9], E[9];
                mmd(C, U + (s * 4 + mu) * 9, Om);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) A[i * 3 + j] = cadd(conjx(Om[j * 3 + i]), (cx){-Om[i * 3 + j].re, -Om[i * 3 + j].im});
                const cx tr = cadd(cadd(A[0], A[4]), A[8]);
                /* X = i Q = i ((i/2) A - (i/6) tr(A) 1) = -(1/2) A + (1/6) tr(A) 1 */
                for (int i = 0; i < 9; ++i) {
                    X[i].re = -0.5 * A[i].re;
                    X[i].im = -0.5 * A[i].im;
                }
                for (int i = 0; i < 3; ++i) {
                    X[i * 4].re += tr.re / 6.0;
                    X[i * 4].im += tr.im / 6.0;
                }
                expm3(X, E);
                mm(E, U + (s * 4 + mu) * 9, W + (s * 4 + mu) * 9);
            }
        }
        memcpy(U, W, sizeof(cx) * 36 * V);
    }
    free(W);
}
