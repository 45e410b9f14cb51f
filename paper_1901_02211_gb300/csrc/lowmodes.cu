// Low modes of H_W = gamma_5 D_W, treated exactly in the sign function.
//
// The paper evaluates eps(H_W) with the Zolotarev rational on the whole
// spectrum (Eq. 4); it mentions low modes only of the overlap operator, for a
// cost comparison (end of Sec. 3).  Overlap codes commonly split off the
// lowest eigenmodes of H_W:
//
//   eps(H) = sum_{j<k} sign(lambda_j) v_j v_j^dag + H R(H^2) P_perp,
//   P_perp = 1 - sum_{j<k} v_j v_j^dag,
//
// so R only needs the interval above lambda_{k+1}^2 and the Krylov solves see
// b_perp = P_perp b, whose spectrum starts there.  The SMP estimate (Eq. 16)
// becomes the usual contraction of gamma_5 D_W y with y = R(H^2) b_perp plus
// the low-mode term 1/2 sum_{alpha,a} sum_j sign(lambda_j) v_j(x) (v_j^dag b).
//
// Eigen-solver: Chebyshev-filtered subspace iteration (Zhou and Saad, 2007)
// on H^2 with a block of m vectors, using the batched FP64 D_W of dslash.cu:
//   filter  Y <- p_d(H^2) Y, p_d the degree-d Chebyshev polynomial that is
//           bounded on [cut, upper] (cut = largest Ritz value of H^2 in the
//           block, upper = the context's spectral upper bound), three-term
//           recurrence with the scaling of Zhou and Saad;
//   orthonormalise  Cholesky QR three times, the first with a small diagonal
//           shift if the Gram matrix is numerically singular;
//   Rayleigh-Ritz first with H^2 on the whole block (its Ritz values bound
//           the filter), then with H on the k + 1 lowest Ritz vectors, which
//           gives the signed eigenvalues; the small Hermitian matrices are
//           diagonalised on the host (cyclic complex Jacobi);
//   stop when those k + 1 pairs have ||H y - lambda y|| <= tol.
// The block lives in the solver's tiled layout with tile width 12.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <numeric>
#include <vector>

#include "smpq_internal.cuh"

namespace {

typedef std::complex<double> cd;

constexpr int LM_MAXM = 48;                                     // block columns
constexpr int LM_GB = 256;                                      // blocks of the Gram kernels
constexpr int LM_GT = 256;                                      // their threads
constexpr int LM_PPT = (LM_MAXM * LM_MAXM + LM_GT - 1) / LM_GT; // pairs per thread

__device__ __forceinline__ size_t tix(int s, int c, int j, int V, int BC) {
    return (((size_t)(j / BC) * V + s) * 12 + c) * BC + (j % BC);
}

__global__ void k_lm_random(double2 *Y, size_t n, unsigned long long seed) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1); // splitmix64
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    unsigned long long w = z * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    w = (w ^ (w >> 30)) * 0xBF58476D1CE4E5B9ull;
    w = (w ^ (w >> 27)) * 0x94D049BB133111EBull;
    w ^= w >> 31;
    Y[i] = make_double2(((z >> 11) + 0.5) * (1.0 / 9007199254740992.0) - 0.5,
                        ((w >> 11) + 0.5) * (1.0 / 9007199254740992.0) - 0.5);
}

// out = a (Z - c Y) + b P   (P nullable)
__global__ void k_lm_cheb(double2 *__restrict__ out, const double2 *__restrict__ Z, const double2 *__restrict__ Y,
                          const double2 *__restrict__ P, size_t n, double a, double c, double b) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 z = Z[i], y = Y[i];
    double2 r = make_double2(a * (z.x - c * y.x), a * (z.y - c * y.y));
    if (P) {
        double2 p = P[i];
        r.x += b * p.x;
        r.y += b * p.y;
    }
    out[i] = r;
}

// part[block][i * my + j] = sum over this block's sites of conj(X_i) (gamma_5 if g5) Y_j
__global__ void __launch_bounds__(LM_GT) k_lm_gram(const double2 *__restrict__ X, int mx, int bcx,
                                                   const double2 *__restrict__ Y, int my, int bcy, int V, int g5,
                                                   double2 *__restrict__ part) {
    __shared__ double2 xs[12 * LM_MAXM], ys[12 * LM_MAXM];
    const int np = mx * my;
    double2 acc[LM_PPT];
#pragma unroll
    for (int q = 0; q < LM_PPT; ++q) acc[q] = make_double2(0, 0);
    for (int s = blockIdx.x; s < V; s += gridDim.x) {
        __syncthreads();
        for (int t = threadIdx.x; t < 12 * mx; t += blockDim.x) xs[t] = X[tix(s, t / mx, t % mx, V, bcx)];
        for (int t = threadIdx.x; t < 12 * my; t += blockDim.x) {
            const int c = t / my;
            double2 v = Y[tix(s, c, t % my, V, bcy)];
            if (g5 && c >= 6) v = make_double2(-v.x, -v.y);
            ys[t] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < LM_PPT; ++q) {
            const int p = threadIdx.x + q * LM_GT;
            if (p < np) {
                const int i = p / my, j = p % my;
#pragma unroll
                for (int c = 0; c < 12; ++c) acc[q] = cfmac(xs[c * mx + i], ys[c * my + j], acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < LM_PPT; ++q) {
        const int p = threadIdx.x + q * LM_GT;
        if (p < np) part[(size_t)blockIdx.x * np + p] = acc[q];
    }
}

// out[p] = sum_b part[b][p] in block order (deterministic)
__global__ void k_lm_sum(const double2 *__restrict__ part, int nb, int np, double2 *__restrict__ out) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double2 a = make_double2(0, 0);
    for (int b = 0; b < nb; ++b) {
        double2 v = part[(size_t)b * np + p];
        a.x += v.x;
        a.y += v.y;
    }
    out[p] = a;
}

// out(s,c,j) = beta base(s,c,j) + alpha (gamma_5 if g5) sum_{i<mx} X(s,c,i) M[i * mo + j]
// (out: mo columns in tiles of bco; X: tiles of bcx).  out may alias base.
__global__ void k_lm_rotate(double2 *out, int mo, int bco, const double2 *base, double beta, double alpha,
                            const double2 *__restrict__ X, int mx, int bcx, const double2 *__restrict__ M, int V,
                            int g5) {
    size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (idx >= (size_t)V * 12 * mo) return;
    const int j = (int)(idx % mo);
    const size_t r = idx / mo;
    const int c = (int)(r % 12), s = (int)(r / 12);
    double2 a = make_double2(0, 0);
    for (int i = 0; i < mx; ++i) a = cfma(X[tix(s, c, i, V, bcx)], M[(size_t)i * mo + j], a);
    double f = alpha * ((g5 && c >= 6) ? -1.0 : 1.0);
    const size_t o = tix(s, c, j, V, bco);
    double2 res = make_double2(f * a.x, f * a.y);
    if (base) {
        double2 bv = base[o];
        res.x += beta * bv.x;
        res.y += beta * bv.y;
    }
    out[o] = res;
}

// part[block][j].x = sum over this block's sites of |gamma_5 T_j - theta_j Y_j|^2 (j < m)
__global__ void k_lm_resid(const double2 *__restrict__ T, const double2 *__restrict__ Y,
                           const double *__restrict__ theta, int m, int V, double2 *__restrict__ part) {
    const int j = threadIdx.x;
    if (j >= m) return;
    const double th = theta[j];
    double a = 0;
    for (int s = blockIdx.x; s < V; s += gridDim.x)
        for (int c = 0; c < 12; ++c) {
            const size_t o = tix(s, c, j, V, 12);
            double2 t = T[o], y = Y[o];
            double f = c >= 6 ? -1.0 : 1.0;
            double dx = f * t.x - th * y.x, dy = f * t.y - th * y.y;
            a += dx * dx + dy * dy;
        }
    part[(size_t)blockIdx.x * m + j] = make_double2(a, 0);
}

// w[(cl * 12 + comp) * k + i] = v_i^dag b_{cl,comp} = sum over the sites of class cl of conj(v_i(site, comp))
__global__ void k_lm_wclass(const double2 *__restrict__ Y, int V, int k, const int *__restrict__ members, int nmem,
                            int ncl, double2 *__restrict__ w) {
    long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)ncl * 12 * k) return;
    const int i = (int)(idx % k), comp = (int)((idx / k) % 12), cl = (int)(idx / (12L * k));
    double2 a = make_double2(0, 0);
    for (int m = 0; m < nmem; ++m) {
        double2 v = Y[tix(members[(size_t)cl * nmem + m], comp, i, V, 12)];
        a.x += v.x;
        a.y -= v.y;
    }
    w[idx] = a;
}

// tiled source b_perp(s, c, j) = [colour(s) == cl_j and c == comp_j] - sum_i v_i(s, c) w[cl_j, comp_j, i]
__global__ void k_lm_source(double2 *__restrict__ b, int B, int BC, int V, const int *__restrict__ colour,
                            const int *__restrict__ rhs_class, const int *__restrict__ src_comp,
                            const double2 *__restrict__ Y, int k, const double2 *__restrict__ w) {
    long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)V * 12 * B) return;
    const int jj = (int)(idx % BC);
    long r = idx / BC;
    const int c = (int)(r % 12);
    r /= 12;
    const int s = (int)(r % V), j = (int)(r / V) * BC + jj;
    const int cl = rhs_class[j];
    if (cl < 0) {
        b[idx] = make_double2(0, 0);
        return;
    }
    const int comp = src_comp[j];
    double2 v = make_double2((colour[s] == cl && c == comp) ? 1.0 : 0.0, 0.0);
    const double2 *wc = w + ((size_t)cl * 12 + comp) * k;
    for (int i = 0; i < k; ++i) {
        double2 p = cmul(Y[tix(s, c, i, V, 12)], wc[i]);
        v.x -= p.x;
        v.y -= p.y;
    }
    b[idx] = v;
}

// y(entry e, c, j) += c0 b_perp(site of entry e, c, j)   (star support layout)
__global__ void k_lm_add_c0b(int n_sup, int B, int BC, int V, const int *__restrict__ supsite,
                             const int *__restrict__ rhs_class, const double2 *__restrict__ bperp, double c0,
                             double2 *__restrict__ y) {
    long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)n_sup * 12 * B) return;
    const int j = (int)(idx % B);
    const long r = idx / B;
    const int c = (int)(r % 12), e = (int)(r / 12);
    const int cl = rhs_class[j];
    if (cl < 0) return;
    const int site = supsite ? supsite[(size_t)cl * n_sup + e] : e;
    const double2 bv = bperp[tix(site, c, j, V, BC)];
    const size_t o = (((size_t)(j / BC) * n_sup + e) * 12 + c) * BC + (j % BC);
    y[o].x += c0 * bv.x;
    y[o].y += c0 * bv.y;
}

// qterm[(cl * 12 + comp) * nmem + m] += sum_i sign_i v_i(x_m, comp) w[cl, comp, i]
__global__ void k_lm_qterm(const int *__restrict__ classes, int nc, const int *__restrict__ members, int nmem,
                           const double2 *__restrict__ Y, int V, int k, const double *__restrict__ sgn,
                           const double2 *__restrict__ w, double2 *__restrict__ qterm) {
    long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (idx >= (long)nc * 12 * nmem) return;
    const int m = (int)(idx % nmem), comp = (int)((idx / nmem) % 12), cl = classes[idx / (12L * nmem)];
    const int x = members[(size_t)cl * nmem + m];
    const double2 *wc = w + ((size_t)cl * 12 + comp) * k;
    double2 a = make_double2(0, 0);
    for (int i = 0; i < k; ++i) {
        double2 p = cmul(Y[tix(x, comp, i, V, 12)], wc[i]);
        a.x += sgn[i] * p.x;
        a.y += sgn[i] * p.y;
    }
    double2 &q = qterm[((size_t)cl * 12 + comp) * nmem + m];
    q.x += a.x;
    q.y += a.y;
}

unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------ host dense linear algebra (m <= 48)
// Cholesky A = L L^dag of a Hermitian matrix (row-major m x m); false if not positive definite.
bool cholesky(std::vector<cd> &A, int m) {
    for (int j = 0; j < m; ++j) {
        double d = A[j * m + j].real();
        for (int p = 0; p < j; ++p) d -= std::norm(A[j * m + p]);
        if (!(d > 0)) return false;
        const double l = std::sqrt(d);
        A[j * m + j] = l;
        for (int i = j + 1; i < m; ++i) {
            cd s = A[i * m + j];
            for (int p = 0; p < j; ++p) s -= A[i * m + p] * std::conj(A[j * m + p]);
            A[i * m + j] = s / l;
        }
        for (int i = 0; i < j; ++i) A[i * m + j] = 0;
    }
    return true;
}

// M = L^{-dag} (upper triangular) for lower triangular L
std::vector<cd> inv_lower_dag(const std::vector<cd> &L, int m) {
    std::vector<cd> X(m * m, 0.0); // X = L^{-1}, lower triangular
    for (int j = 0; j < m; ++j) {
        X[j * m + j] = 1.0 / L[j * m + j];
        for (int i = j + 1; i < m; ++i) {
            cd s = 0;
            for (int p = j; p < i; ++p) s += L[i * m + p] * X[p * m + j];
            X[i * m + j] = -s / L[i * m + i];
        }
    }
    std::vector<cd> M(m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) M[i * m + j] = std::conj(X[j * m + i]);
    return M;
}

// Cyclic Jacobi for a Hermitian matrix A (row-major, overwritten): eigenvalues
// in w, eigenvectors in the columns of Z.  Each rotation first turns the (p, q)
// element real with a phase on column/row q, then applies the real symmetric
// Jacobi rotation that annihilates it.
void jacobi_eig(std::vector<cd> A, int m, std::vector<double> &w, std::vector<cd> &Z) {
    Z.assign(m * m, 0.0);
    for (int i = 0; i < m; ++i) Z[i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double a = std::norm(A[i * m + j]);
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-30 * tot || off == 0) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                const cd apq = A[p * m + q];
                const double r = std::abs(apq);
                if (r <= 1e-300) continue;
                const cd u = apq / r; // A_pq = r u
                const double app = A[p * m + p].real(), aqq = A[q * m + q].real();
                const double tau = (aqq - app) / (2 * r);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
                const double c = 1 / std::sqrt(1 + t * t), s = t * c;
                // unitary G on (p, q): columns p' = c e_p - s conj(u) e_q, q' = s e_p + c conj(u) e_q
                const cd gpp = c, gqp = -s * std::conj(u), gpq = s, gqq = c * std::conj(u);
                for (int i = 0; i < m; ++i) { // A <- A G
                    const cd aip = A[i * m + p], aiq = A[i * m + q];
                    A[i * m + p] = aip * gpp + aiq * gqp;
                    A[i * m + q] = aip * gpq + aiq * gqq;
                }
                for (int i = 0; i < m; ++i) { // A <- G^dag A
                    const cd api = A[p * m + i], aqi = A[q * m + i];
                    A[p * m + i] = std::conj(gpp) * api + std::conj(gqp) * aqi;
                    A[q * m + i] = std::conj(gpq) * api + std::conj(gqq) * aqi;
                }
                A[p * m + q] = A[q * m + p] = 0;
                for (int i = 0; i < m; ++i) { // Z <- Z G
                    const cd zip = Z[i * m + p], ziq = Z[i * m + q];
                    Z[i * m + p] = zip * gpp + ziq * gqp;
                    Z[i * m + q] = zip * gpq + ziq * gqq;
                }
            }
    }
    w.resize(m);
    for (int i = 0; i < m; ++i) w[i] = A[i * m + i].real();
}

std::vector<cd> hermitian_part(const std::vector<cd> &G, int m) {
    std::vector<cd> H(G);
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j) {
            cd a = 0.5 * (G[i * m + j] + std::conj(G[j * m + i]));
            H[i * m + j] = a;
            H[j * m + i] = std::conj(a);
        }
    return H;
}

struct Eig {
    smpq_ctx *ctx;
    cudaStream_t st;
    int V, m;
    size_t n; // complex entries of one block
    double2 *Y, *T, *Z, *A, *Bq, *part, *sum, *mat;
    double *theta;

    int gram(const double2 *X, int mx, int bcx, const double2 *Yv, int my, int bcy, int g5, std::vector<cd> &G) {
        k_lm_gram<<<LM_GB, LM_GT, 0, st>>>(X, mx, bcx, Yv, my, bcy, V, g5, part);
        k_lm_sum<<<nblk(mx * my), 256, 0, st>>>(part, LM_GB, mx * my, sum);
        G.resize((size_t)mx * my);
        cudaMemcpyAsync(G.data(), sum, G.size() * sizeof(cd), cudaMemcpyDeviceToHost, st);
        ctx->launches += 2;
        return cuda_check(ctx, cudaStreamSynchronize(st), "low-mode Gram matrix");
    }
    // out = X M (m x m), out-of-place
    void rotate(double2 *out, const double2 *X, const std::vector<cd> &M) {
        cudaMemcpyAsync(mat, M.data(), M.size() * sizeof(cd), cudaMemcpyHostToDevice, st);
        k_lm_rotate<<<nblk(n), 256, 0, st>>>(out, m, 12, nullptr, 0.0, 1.0, X, m, 12, mat, V, 0);
        ctx->launches += 1;
    }
    void h2(const double2 *in, double2 *out) { // out = D_W^dag D_W in, via T
        launch_dslash<double>(ctx->geom, ctx->U64.p, in, T, m, 12, 0, ctx->opt.kappa, st);
        launch_dslash<double>(ctx->geom, ctx->U64.p, T, out, m, 12, 1, ctx->opt.kappa, st);
        ctx->launches += 2;
    }
    // Y <- Y R with Y^dag Y = 1 (Cholesky QR, three passes)
    int orthonormalise() {
        for (int pass = 0; pass < 3; ++pass) {
            std::vector<cd> G;
            int rc = gram(Y, m, 12, Y, m, 12, 0, G);
            if (rc) return rc;
            for (int i = 0; i < m; ++i) G[i * m + i] = G[i * m + i].real();
            std::vector<cd> L = G;
            if (!cholesky(L, m)) {
                double tr = 0;
                for (int i = 0; i < m; ++i) tr += G[i * m + i].real();
                L = G;
                for (int i = 0; i < m; ++i) L[i * m + i] += 1e-13 * tr;
                if (!cholesky(L, m))
                    return set_err(ctx, SMPQ_EBREAKDOWN, "low modes: the block lost rank (Cholesky QR failed)");
            }
            rotate(A, Y, inv_lower_dag(L, m));
            std::swap(Y, A);
        }
        return SMPQ_OK;
    }
    // Rayleigh-Ritz in two stages.  (1) With H^2 = (D_W Y)^dag (D_W Y) on the
    // whole block: Ritz values th2 ascending (upper bounds of the lowest
    // eigenvalues of H^2, so no spurious small ones).  (2) With H on the K
    // lowest of those vectors: signed eigenvalues lam ordered by |lam| and the
    // residual norms ||H y - lam y||.  (Rayleigh-Ritz with the indefinite H on
    // the whole block yields spurious Ritz values near 0 from unconverged
    // directions that mix +lambda and -lambda.)  Afterwards Y holds the Ritz
    // vectors and T = D_W Y.
    int rayleigh_ritz(int K, std::vector<double> &th2, std::vector<double> &lam, std::vector<double> &res) {
        launch_dslash<double>(ctx->geom, ctx->U64.p, Y, T, m, 12, 0, ctx->opt.kappa, st);
        ctx->launches += 1;
        std::vector<cd> G;
        int rc = gram(T, m, 12, T, m, 12, 0, G);
        if (rc) return rc;
        std::vector<double> w;
        std::vector<cd> Zm;
        jacobi_eig(hermitian_part(G, m), m, w, Zm);
        std::vector<int> ord(m);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return w[a] < w[b]; });
        std::vector<cd> Zs(m * m);
        th2.resize(m);
        for (int j = 0; j < m; ++j) {
            th2[j] = w[ord[j]];
            for (int i = 0; i < m; ++i) Zs[i * m + j] = Zm[i * m + ord[j]];
        }
        rotate(A, Y, Zs);
        std::swap(Y, A);
        rotate(Bq, T, Zs);
        std::swap(T, Bq);
        // stage 2 on the first K columns
        if ((rc = gram(Y, K, 12, T, K, 12, 1, G))) return rc;
        jacobi_eig(hermitian_part(G, K), K, w, Zm);
        ord.resize(K);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return std::fabs(w[a]) < std::fabs(w[b]); });
        std::fill(Zs.begin(), Zs.end(), cd(0.0));
        for (int j = K; j < m; ++j) Zs[j * m + j] = 1.0;
        lam.resize(K);
        for (int j = 0; j < K; ++j) {
            lam[j] = w[ord[j]];
            for (int i = 0; i < K; ++i) Zs[i * m + j] = Zm[i * K + ord[j]];
        }
        rotate(A, Y, Zs);
        std::swap(Y, A);
        rotate(Bq, T, Zs);
        std::swap(T, Bq);
        cudaMemcpyAsync(theta, lam.data(), K * sizeof(double), cudaMemcpyHostToDevice, st);
        k_lm_resid<<<LM_GB, 64, 0, st>>>(T, Y, theta, K, V, part);
        k_lm_sum<<<1, 64, 0, st>>>(part, LM_GB, K, sum);
        ctx->launches += 2;
        std::vector<cd> r(K);
        cudaMemcpyAsync(r.data(), sum, K * sizeof(cd), cudaMemcpyDeviceToHost, st);
        rc = cuda_check(ctx, cudaStreamSynchronize(st), "low-mode residuals");
        if (rc) return rc;
        res.resize(K);
        for (int j = 0; j < K; ++j) res[j] = std::sqrt(std::max(0.0, r[j].real()));
        return SMPQ_OK;
    }
    // Y <- p_d(H^2) Y: scaled Chebyshev recurrence damping [cut, upper], normalised near lo
    void filter(int d, double lo, double cut, double upper) {
        const double e = 0.5 * (upper - cut), c = 0.5 * (upper + cut);
        double sigma = e / (lo - c);
        const double sigma1 = sigma;
        double2 *Y0 = Y, *Y1 = A, *Y2 = Bq;
        h2(Y0, Z);
        k_lm_cheb<<<nblk(n), 256, 0, st>>>(Y1, Z, Y0, nullptr, n, sigma1 / e, c, 0.0);
        ctx->launches += 1;
        for (int i = 2; i <= d; ++i) {
            const double sn = 1.0 / (2.0 / sigma1 - sigma);
            h2(Y1, Z);
            k_lm_cheb<<<nblk(n), 256, 0, st>>>(Y2, Z, Y1, Y0, n, 2.0 * sn / e, c, -sigma * sn);
            ctx->launches += 1;
            double2 *t = Y0;
            Y0 = Y1;
            Y1 = Y2;
            Y2 = t;
            sigma = sn;
        }
        // the filtered block is in Y1; keep the three buffers distinct
        double2 *bufs[3] = {Y, A, Bq};
        double2 *rest[2];
        int r = 0;
        for (double2 *b : bufs)
            if (b != Y1) rest[r++] = b;
        Y = Y1;
        A = rest[0];
        Bq = rest[1];
    }
};

} // namespace

void lowmodes_clear(smpq_ctx *ctx) {
    release(ctx->lm_vec);
    release(ctx->lm_sgn);
    release(ctx->lm_w);
    ctx->lm_k = ctx->lm_m = 0;
    ctx->lm_val.clear();
}

int lowmodes_compute(smpq_ctx *ctx, int k, int m, double tol, int max_iter, int degree, double *evals,
                     double *resid, int *iterations) {
    if (m % 12 || m < 12 || m > LM_MAXM || k < 1 || k + 1 > m)
        return set_err(ctx, SMPQ_EINVAL, "low modes: need 1 <= k < block, block a multiple of 12 and at most 48");
    lowmodes_clear(ctx);
    cudaStream_t st = ctx->stream;
    const int V = ctx->V;
    const size_t n = (size_t)V * 12 * m;
    Buf scr;
    const size_t parts = (size_t)LM_GB * m * m;
    int rc = ensure(ctx, scr, (5 * n + parts + 2 * (size_t)m * m) * sizeof(double2) + m * sizeof(double));
    if (rc) return rc;
    Eig E;
    E.ctx = ctx;
    E.st = st;
    E.V = V;
    E.m = m;
    E.n = n;
    double2 *p = (double2 *)scr.p;
    E.Y = p;
    E.T = p + n;
    E.Z = p + 2 * n;
    E.A = p + 3 * n;
    E.Bq = p + 4 * n;
    E.part = p + 5 * n;
    E.sum = E.part + parts;
    E.mat = E.sum + (size_t)m * m;
    E.theta = (double *)(E.mat + (size_t)m * m);
    k_lm_random<<<nblk(n), 256, 0, st>>>(E.Y, n, 0x10f3a0d5ull);
    ctx->launches += 1;
    const int K = k + 1;
    std::vector<double> th2, lam, res;
    int it = 0;
    rc = E.orthonormalise();
    if (!rc) rc = E.rayleigh_ritz(K, th2, lam, res);
    const double upper = ctx->lmax2;
    while (!rc) {
        bool done = true;
        for (int j = 0; j < K; ++j) done = done && res[j] <= tol;
        if (done) break;
        if (it >= max_iter) {
            rc = set_err(ctx, SMPQ_ENOCONV, "low modes: not converged in " + std::to_string(max_iter) + " filter steps");
            break;
        }
        const double cut = th2[m - 1];
        double lo = th2[0];
        if (!(cut < upper)) {
            rc = set_err(ctx, SMPQ_EINVAL, "low modes: the block's Ritz values reach the spectral upper bound");
            break;
        }
        if (!(lo < 0.9 * cut)) lo = 0;
        E.filter(degree, lo, cut, upper);
        rc = E.orthonormalise();
        if (!rc) rc = E.rayleigh_ritz(K, th2, lam, res);
        ++it;
    }
    if (!rc) {
        rc = ensure(ctx, ctx->lm_vec, n * sizeof(double2));
        if (!rc) rc = ensure(ctx, ctx->lm_sgn, k * sizeof(double));
    }
    if (!rc) {
        cudaMemcpyAsync(ctx->lm_vec.p, E.Y, n * sizeof(double2), cudaMemcpyDeviceToDevice, st);
        std::vector<double> sg(k);
        for (int j = 0; j < k; ++j) sg[j] = lam[j] >= 0 ? 1.0 : -1.0;
        cudaMemcpyAsync(ctx->lm_sgn.p, sg.data(), k * sizeof(double), cudaMemcpyHostToDevice, st);
        rc = cuda_check(ctx, cudaStreamSynchronize(st), "low modes");
    }
    if (!rc) {
        ctx->lm_k = k;
        ctx->lm_m = m;
        ctx->lm_val = lam;
        if (evals) std::copy(lam.begin(), lam.end(), evals);
        if (resid) std::copy(res.begin(), res.end(), resid);
        if (iterations) *iterations = it;
    } else {
        lowmodes_clear(ctx);
    }
    cudaStreamSynchronize(st);
    release(scr);
    return rc;
}

int lowmodes_class_overlaps(smpq_ctx *ctx, cudaStream_t st) {
    const int k = ctx->lm_k;
    const size_t nw = (size_t)ctx->n_classes * 12 * k;
    int rc = ensure(ctx, ctx->lm_w, nw * sizeof(double2));
    if (rc) return rc;
    k_lm_wclass<<<nblk(nw), 256, 0, st>>>((const double2 *)ctx->lm_vec.p, ctx->V, k, (const int *)ctx->d_members.p,
                                          ctx->members, ctx->n_classes, (double2 *)ctx->lm_w.p);
    ctx->launches += 1;
    return SMPQ_OK;
}

void lowmodes_source(smpq_ctx *ctx, double2 *bperp, int B, int BC, const int *d_rhs_class, const int *d_src_comp,
                     cudaStream_t st) {
    const size_t n = (size_t)ctx->V * 12 * B;
    k_lm_source<<<nblk(n), 256, 0, st>>>(bperp, B, BC, ctx->V, (const int *)ctx->d_colour.p, d_rhs_class, d_src_comp,
                                         (const double2 *)ctx->lm_vec.p, ctx->lm_k, (const double2 *)ctx->lm_w.p);
    ctx->launches += 1;
}

void lowmodes_add_c0b(smpq_ctx *ctx, int n_sup, int B, int BC, const int *d_supsite, const int *d_rhs_class,
                      const double2 *bperp, double2 *y, cudaStream_t st) {
    const size_t n = (size_t)n_sup * 12 * B;
    k_lm_add_c0b<<<nblk(n), 256, 0, st>>>(n_sup, B, BC, ctx->V, d_supsite, d_rhs_class, bperp, ctx->c0, y);
    ctx->launches += 1;
}

void lowmodes_qterm(smpq_ctx *ctx, const int *d_classes, int nc, double2 *qterm, cudaStream_t st) {
    const size_t n = (size_t)nc * 12 * ctx->members;
    k_lm_qterm<<<nblk(n), 256, 0, st>>>(d_classes, nc, (const int *)ctx->d_members.p, ctx->members,
                                        (const double2 *)ctx->lm_vec.p, ctx->V, ctx->lm_k,
                                        (const double *)ctx->lm_sgn.p, (const double2 *)ctx->lm_w.p, qterm);
    ctx->launches += 1;
}

int lowmodes_dov_project(smpq_ctx *ctx, const double2 *b, double2 *bperp, int B, std::vector<double> &wd,
                         cudaStream_t st) {
    const int k = ctx->lm_k, V = ctx->V;
    const size_t parts = (size_t)LM_GB * k * LM_MAXM;
    int rc = ensure(ctx, ctx->lm_w, (parts + (size_t)k * LM_MAXM + (size_t)k * B) * sizeof(double2));
    if (rc) return rc;
    double2 *part = (double2 *)ctx->lm_w.p, *sum = part + parts, *mat = sum + (size_t)k * LM_MAXM;
    const double2 *Y = (const double2 *)ctx->lm_vec.p;
    std::vector<cd> W((size_t)k * B); // W[i * B + j] = v_i^dag b_j
    for (int j0 = 0; j0 < B; j0 += LM_MAXM) {
        const int nb = std::min(LM_MAXM, B - j0);
        k_lm_gram<<<LM_GB, LM_GT, 0, st>>>(Y, k, 12, b + (size_t)j0 * V * 12, nb, 1, V, 0, part);
        k_lm_sum<<<nblk(k * nb), 256, 0, st>>>(part, LM_GB, k * nb, sum);
        std::vector<cd> g((size_t)k * nb);
        cudaMemcpyAsync(g.data(), sum, g.size() * sizeof(cd), cudaMemcpyDeviceToHost, st);
        if ((rc = cuda_check(ctx, cudaStreamSynchronize(st), "low-mode overlaps"))) return rc;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < nb; ++j) W[(size_t)i * B + j0 + j] = g[(size_t)i * nb + j];
        ctx->launches += 2;
    }
    cudaMemcpyAsync(mat, W.data(), W.size() * sizeof(cd), cudaMemcpyHostToDevice, st);
    k_lm_rotate<<<nblk((size_t)V * 12 * B), 256, 0, st>>>(bperp, B, 1, b, 1.0, -1.0, Y, k, 12, mat, V, 0);
    ctx->launches += 1;
    wd.resize(2 * W.size());
    std::memcpy(wd.data(), W.data(), W.size() * sizeof(cd));
    return cuda_check(ctx, cudaStreamSynchronize(st), "low-mode projection");
}

int lowmodes_dov_finish(smpq_ctx *ctx, double2 *out, int B, const std::vector<double> &wd, cudaStream_t st) {
    const int k = ctx->lm_k, V = ctx->V;
    const size_t parts = (size_t)LM_GB * k * LM_MAXM;
    double2 *mat = (double2 *)ctx->lm_w.p + parts + (size_t)k * LM_MAXM;
    std::vector<cd> M((size_t)k * B);
    for (int i = 0; i < k; ++i) {
        const double s = ctx->lm_val[i] >= 0 ? 1.0 : -1.0;
        for (int j = 0; j < B; ++j) M[(size_t)i * B + j] = s * cd(wd[2 * ((size_t)i * B + j)], wd[2 * ((size_t)i * B + j) + 1]);
    }
    cudaMemcpyAsync(mat, M.data(), M.size() * sizeof(cd), cudaMemcpyHostToDevice, st);
    k_lm_rotate<<<nblk((size_t)V * 12 * B), 256, 0, st>>>(out, B, 1, out, 1.0, 1.0, (const double2 *)ctx->lm_vec.p, k,
                                                          12, mat, V, 1);
    ctx->launches += 1;
    return cuda_check(ctx, cudaStreamSynchronize(st), "low-mode term of D_ov");
}
