/* CPU FP64 oracle, compiled part.  TEST INFRASTRUCTURE ONLY: used by the test
 * suite, the smoke check and the benchmark's CPU-baseline leg, never by the
 * product path.  Plain loops (OpenMP over sites), written for checkability.
 *
 * It restates, in C, the same steps as oracle/dirac.py and oracle/msolve.py:
 *   D_W psi(x) = psi(x) - kappa sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                      + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)]
 *   (Sec. 2.1, around Eq. 3), H = gamma_5 D_W, H^2 = D_W^dag D_W (Eq. 4), and
 *   the multi-shift CG for (H^2 + q_i) x_i = b (Eqs. 6-8).
 * Chiral basis: gamma_k = [[0,-i sigma_k],[i sigma_k,0]], gamma_4 = [[0,1],[1,0]],
 * gamma_5 = diag(1,1,-1,-1).
 *
 * Layouts (complex numbers as interleaved re, im doubles):
 *   U   [V][4][3][3]          link U_mu(x), row-major colour
 *   psi [V][4][3][B]          site, spin, colour, right-hand side (B fastest)
 *   x   [n_shift][V][4][3][B]
 */
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static cplx G[4][4][4]; /* gamma_mu, mu = 0..3 (x, y, z, t) */
static int g_init = 0;

static void init_gamma(void) {
    if (g_init) return;
    memset(G, 0, sizeof(G));
    /* sigma matrices */
    cplx s[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                G[k][i][2 + j] = -I * s[k][i][j];
                G[k][2 + i][j] = I * s[k][i][j];
            }
    G[3][0][2] = G[3][1][3] = G[3][2][0] = G[3][3][1] = 1;
    g_init = 1;
}

typedef struct {
    int dims[4];
    long V;
    long *fwd; /* [4][V] */
    long *bwd;
    double *sf; /* boundary factor of the forward hop [4][V] */
    double *sb;
} lat_t;

static void lat_build(lat_t *L, const int dims[4], const int bc[4]) {
    memcpy(L->dims, dims, sizeof(int) * 4);
    L->V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    L->fwd = malloc(sizeof(long) * 4 * L->V);
    L->bwd = malloc(sizeof(long) * 4 * L->V);
    L->sf = malloc(sizeof(double) * 4 * L->V);
    L->sb = malloc(sizeof(double) * 4 * L->V);
    for (long s = 0; s < L->V; ++s) {
        int c[4];
        long r = s;
        for (int mu = 0; mu < 4; ++mu) { c[mu] = r % dims[mu]; r /= dims[mu]; }
        for (int mu = 0; mu < 4; ++mu) {
            int cf[4], cb[4];
            memcpy(cf, c, sizeof(c));
            memcpy(cb, c, sizeof(c));
            cf[mu] = (c[mu] + 1) % dims[mu];
            cb[mu] = (c[mu] - 1 + dims[mu]) % dims[mu];
            long f = cf[0] + (long)dims[0] * (cf[1] + (long)dims[1] * (cf[2] + (long)dims[2] * cf[3]));
            long b = cb[0] + (long)dims[0] * (cb[1] + (long)dims[1] * (cb[2] + (long)dims[2] * cb[3]));
            L->fwd[mu * L->V + s] = f;
            L->bwd[mu * L->V + s] = b;
            L->sf[mu * L->V + s] = (c[mu] == dims[mu] - 1) ? bc[mu] : 1.0;
            L->sb[mu * L->V + s] = (c[mu] == 0) ? bc[mu] : 1.0;
        }
    }
}

static void lat_free(lat_t *L) {
    free(L->fwd); free(L->bwd); free(L->sf); free(L->sb);
}

/* out = D_W in, B right-hand sides; optional gamma_5 on the result. */
static void dslash(const lat_t *L, const cplx *U, const cplx *in, cplx *out, double kappa, int B, int g5out) {
    init_gamma();
    long V = L->V;
#pragma omp parallel
    {
        cplx *t = malloc(sizeof(cplx) * 12 * B);
#pragma omp for schedule(static)
        for (long s = 0; s < V; ++s) {
            cplx *o = out + s * 12 * B;
            for (int k = 0; k < 12 * B; ++k) o[k] = in[s * 12 * B + k];
            for (int mu = 0; mu < 4; ++mu) {
                for (int dir = 0; dir < 2; ++dir) {
                    long nb = dir == 0 ? L->fwd[mu * V + s] : L->bwd[mu * V + s];
                    double f = dir == 0 ? L->sf[mu * V + s] : L->sb[mu * V + s];
                    const cplx *u = dir == 0 ? U + (s * 4 + mu) * 9 : U + (nb * 4 + mu) * 9;
                    const cplx *p = in + nb * 12 * B;
                    /* t[beta][a][n] = sum_b W_ab p[beta][b][n], W = U or U^dag */
                    for (int beta = 0; beta < 4; ++beta)
                        for (int a = 0; a < 3; ++a)
                            for (int n = 0; n < B; ++n) {
                                cplx acc = 0;
                                for (int b = 0; b < 3; ++b) {
                                    cplx w = dir == 0 ? u[a * 3 + b] : conj(u[b * 3 + a]);
                                    acc += w * p[(beta * 3 + b) * B + n];
                                }
                                t[(beta * 3 + a) * B + n] = f * acc;
                            }
                    double sg = dir == 0 ? -1.0 : 1.0; /* (1 - gamma) forward, (1 + gamma) backward */
                    for (int alpha = 0; alpha < 4; ++alpha)
                        for (int beta = 0; beta < 4; ++beta) {
                            cplx m = (alpha == beta ? 1.0 : 0.0) + sg * G[mu][alpha][beta];
                            if (m == 0) continue;
                            for (int a = 0; a < 3; ++a)
                                for (int n = 0; n < B; ++n)
                                    o[(alpha * 3 + a) * B + n] -= kappa * m * t[(beta * 3 + a) * B + n];
                        }
                }
            }
            if (g5out)
                for (int alpha = 2; alpha < 4; ++alpha)
                    for (int k = 0; k < 3 * B; ++k) o[alpha * 3 * B + k] = -o[alpha * 3 * B + k];
        }
        free(t);
    }
}

/* out = gamma_5 D_W gamma_5 D_W in = H^2 in (tmp: scratch of the same size). */
static void h2(const lat_t *L, const cplx *U, const cplx *in, cplx *out, cplx *tmp, double kappa, int B) {
    dslash(L, U, in, tmp, kappa, B, 1);
    dslash(L, U, tmp, out, kappa, B, 1);
}

/* Per-column Re <u, v>, deterministic: 64 fixed chunks of the index range,
 * each summed in index order, then the chunks added in chunk order. */
#define NCHUNK 64
static void dot_re(const cplx *u, const cplx *v, long N, int B, double *out) {
    double *part = calloc((size_t)NCHUNK * B, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int c = 0; c < NCHUNK; ++c) {
        long lo = N * c / NCHUNK, hi = N * (c + 1) / NCHUNK;
        for (long i = lo; i < hi; ++i)
            for (int n = 0; n < B; ++n) part[c * B + n] += creal(conj(u[i * B + n]) * v[i * B + n]);
    }
    for (int n = 0; n < B; ++n) {
        out[n] = 0;
        for (int c = 0; c < NCHUNK; ++c) out[n] += part[c * B + n];
    }
    free(part);
}

void orc_dslash(const int dims[4], const int bc[4], double kappa, const double *U, const double *in,
                double *out, int B, int g5out) {
    lat_t L;
    lat_build(&L, dims, bc);
    dslash(&L, (const cplx *)U, (const cplx *)in, (cplx *)out, kappa, B, g5out);
    lat_free(&L);
}

void orc_h2(const int dims[4], const int bc[4], double kappa, const double *U, const double *in, double *out,
            int B) {
    lat_t L;
    lat_build(&L, dims, bc);
    long N = 12 * L.V;
    cplx *tmp = malloc(sizeof(cplx) * N * B);
    h2(&L, (const cplx *)U, (const cplx *)in, (cplx *)out, tmp, kappa, B);
    free(tmp);
    lat_free(&L);
}

/* Multi-shift CG, the recurrences of oracle/msolve.py (Frommer et al. 1995;
 * Jegerlehner 1996).  x: [n][N][B] output.  resid: [n][B] final |zeta| ||r||/||b||.
 * Returns the iteration count, or -1 if max_iter was reached. */
int orc_multishift(const int dims[4], const int bc[4], double kappa, const double *Ud, const double *bd, int B,
                   int nshift, const double *shifts, double tol, int max_iter, double *xd, double *resid) {
    lat_t L;
    lat_build(&L, dims, bc);
    const cplx *U = (const cplx *)Ud;
    const cplx *b = (const cplx *)bd;
    cplx *x = (cplx *)xd;
    long N = 12 * L.V;
    long NB = N * B;
    cplx *r = malloc(sizeof(cplx) * NB), *p = malloc(sizeof(cplx) * NB), *Ap = malloc(sizeof(cplx) * NB),
         *tmp = malloc(sizeof(cplx) * NB), *ps = malloc(sizeof(cplx) * NB * nshift);
    double *rr = malloc(sizeof(double) * B), *bb = malloc(sizeof(double) * B), *pAp = malloc(sizeof(double) * B),
           *rrn = malloc(sizeof(double) * B), *alpha = malloc(sizeof(double) * B), *beta = malloc(sizeof(double) * B),
           *alpha_prev = malloc(sizeof(double) * B), *beta_prev = malloc(sizeof(double) * B);
    double *zeta = malloc(sizeof(double) * nshift * B), *zeta_prev = malloc(sizeof(double) * nshift * B),
           *zeta_new = malloc(sizeof(double) * nshift * B), *alpha_s = malloc(sizeof(double) * nshift * B),
           *beta_s = malloc(sizeof(double) * nshift * B);
    unsigned char *act = malloc(nshift * B), *col = malloc(B);
    double s0 = shifts[0];
    for (int i = 1; i < nshift; ++i) s0 = fmin(s0, shifts[i]);

    memset(x, 0, sizeof(cplx) * NB * nshift);
    memcpy(r, b, sizeof(cplx) * NB);
    memcpy(p, b, sizeof(cplx) * NB);
    for (int i = 0; i < nshift; ++i) memcpy(ps + i * NB, b, sizeof(cplx) * NB);
    dot_re(r, r, N, B, rr);
    memcpy(bb, rr, sizeof(double) * B);
    double tol2 = tol * tol;
    for (int n = 0; n < B; ++n) {
        alpha_prev[n] = 1;
        beta_prev[n] = 0;
        for (int i = 0; i < nshift; ++i) {
            zeta[i * B + n] = zeta_prev[i * B + n] = 1;
            act[i * B + n] = rr[n] > tol2 * bb[n];
        }
    }
    int k = 0;
    for (;;) {
        int any = 0;
        for (int n = 0; n < B; ++n) {
            col[n] = 0;
            for (int i = 0; i < nshift; ++i) col[n] |= act[i * B + n];
            any |= col[n];
        }
        if (!any) break;
        if (k >= max_iter) { k = -1; break; }
        h2(&L, U, p, Ap, tmp, kappa, B);
#pragma omp parallel for schedule(static)
        for (long j = 0; j < NB; ++j) Ap[j] += s0 * p[j];
        dot_re(p, Ap, N, B, pAp);
        for (int n = 0; n < B; ++n) {
            alpha[n] = col[n] ? rr[n] / pAp[n] : 0.0;
            for (int i = 0; i < nshift; ++i) {
                int ix = i * B + n;
                if (!act[ix]) { zeta_new[ix] = zeta[ix]; alpha_s[ix] = 0; continue; }
                double sig = shifts[i] - s0;
                double den = alpha[n] * beta_prev[n] * (zeta_prev[ix] - zeta[ix]) +
                             zeta_prev[ix] * alpha_prev[n] * (1.0 + sig * alpha[n]);
                zeta_new[ix] = zeta[ix] * zeta_prev[ix] * alpha_prev[n] / den;
                alpha_s[ix] = alpha[n] * zeta_new[ix] / zeta[ix];
            }
        }
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j)
            for (int n = 0; n < B; ++n) {
                long jj = j * B + n;
                for (int i = 0; i < nshift; ++i) x[i * NB + jj] += alpha_s[i * B + n] * ps[i * NB + jj];
                r[jj] -= alpha[n] * Ap[jj];
            }
        dot_re(r, r, N, B, rrn);
        for (int n = 0; n < B; ++n) {
            beta[n] = col[n] ? rrn[n] / rr[n] : 0.0;
            for (int i = 0; i < nshift; ++i) {
                int ix = i * B + n;
                double q = zeta_new[ix] / zeta[ix];
                beta_s[ix] = beta[n] * q * q;
            }
        }
#pragma omp parallel for schedule(static)
        for (long j = 0; j < N; ++j)
            for (int n = 0; n < B; ++n) {
                long jj = j * B + n;
                for (int i = 0; i < nshift; ++i) {
                    int ix = i * B + n;
                    if (act[ix]) ps[i * NB + jj] = zeta_new[ix] * r[jj] + beta_s[ix] * ps[i * NB + jj];
                }
                if (col[n]) p[jj] = r[jj] + beta[n] * p[jj];
            }
        for (int n = 0; n < B; ++n) {
            for (int i = 0; i < nshift; ++i) {
                int ix = i * B + n;
                if (act[ix]) { zeta_prev[ix] = zeta[ix]; zeta[ix] = zeta_new[ix]; }
            }
            if (col[n]) { alpha_prev[n] = alpha[n]; beta_prev[n] = beta[n]; rr[n] = rrn[n]; }
            for (int i = 0; i < nshift; ++i) {
                int ix = i * B + n;
                act[ix] = act[ix] && (zeta[ix] * zeta[ix] * rr[n] > tol2 * bb[n]);
            }
        }
        ++k;
    }
    for (int i = 0; i < nshift; ++i)
        for (int n = 0; n < B; ++n) resid[i * B + n] = sqrt(zeta[i * B + n] * zeta[i * B + n] * rr[n] / bb[n]);
    free(r); free(p); free(Ap); free(tmp); free(ps);
    free(rr); free(bb); free(pAp); free(rrn); free(alpha); free(beta); free(alpha_prev); free(beta_prev);
    free(zeta); free(zeta_prev); free(zeta_new); free(alpha_s); free(beta_s); free(act); free(col);
    lat_free(&L);
    return k;
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
