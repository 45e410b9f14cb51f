// Symmetric multi-probing colouring (Sec. 2.2, Eq. 19), the star support of
// the shifted vectors, the gamma_5 trace contraction (Eqs. 5, 16) and Q.
//
// Colour numbering (the paper fixes only which sites share a colour):
//   b_mu = x_mu mod r
//   mode 0 (Normal):  c = b_x + r (b_y + r (b_z + r b_t))                   r^4 colours
//   mode 1 (Split):   c = 2 c_normal + (sum_mu floor(x_mu / r)) mod 2       2 r^4 colours
//   mode 2 (Combine): h = r/2, e_mu = b_mu mod h, d_mu = floor(b_mu / h);
//                     if d_x = 1 flip every d_mu (pairs d with 1 - d, i.e. the
//                     set with its (h,h,h,h) translate);
//                     c = 8 (e_x + h (e_y + h (e_z + h e_t))) + d_y + 2 d_z + 4 d_t   r^4 / 2 colours
#include <algorithm>
#include <string>
#include <vector>

#include "smpq_internal.cuh"
#include "wilson.cuh"

int colour_sites_host(const int dims[4], int r, int mode, std::vector<int> &colour, int *n_classes,
                      std::string *why) {
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] < 1 || r < 1 || dims[mu] % r) {
            if (why) *why = "r must divide every lattice extent";
            return SMPQ_EINVAL;
        }
    if (mode < 0 || mode > 2) {
        if (why) *why = "mode must be 0 (normal), 1 (split) or 2 (combine)";
        return SMPQ_EINVAL;
    }
    if (mode == 1)
        for (int mu = 0; mu < 4; ++mu)
            if ((dims[mu] / r) % 2) {
                if (why) *why = "split mode needs an even number of same-colour sites per direction";
                return SMPQ_EINVAL;
            }
    if (mode == 2 && r % 2) {
        if (why) *why = "combine mode needs even r";
        return SMPQ_EINVAL;
    }
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    colour.resize(V);
    const int h = r / 2;
    for (long s = 0; s < V; ++s) {
        int x[4];
        long t = s;
        for (int mu = 0; mu < 4; ++mu) { x[mu] = (int)(t % dims[mu]); t /= dims[mu]; }
        int b[4];
        for (int mu = 0; mu < 4; ++mu) b[mu] = x[mu] % r;
        int c;
        if (mode == 0 || mode == 1) {
            c = b[0] + r * (b[1] + r * (b[2] + r * b[3]));
            if (mode == 1) c = 2 * c + ((x[0] / r + x[1] / r + x[2] / r + x[3] / r) & 1);
        } else {
            int e[4], d[4];
            for (int mu = 0; mu < 4; ++mu) { e[mu] = b[mu] % h; d[mu] = b[mu] / h; }
            if (d[0] == 1)
                for (int mu = 0; mu < 4; ++mu) d[mu] = 1 - d[mu];
            c = 8 * (e[0] + h * (e[1] + h * (e[2] + h * e[3]))) + d[1] + 2 * d[2] + 4 * d[3];
        }
        colour[s] = c;
    }
    int n = mode == 0 ? r * r * r * r : (mode == 1 ? 2 * r * r * r * r : r * r * r * r / 2);
    *n_classes = n;
    return SMPQ_OK;
}

// Star support: entry k = 9 m + d of class c is member m (d = 0) or its
// neighbour in direction mu (d = 1 + 2 mu forward, d = 2 + 2 mu backward).
__global__ void star_kernel(Geom g, const int *__restrict__ members, int n_classes, int nmem, int *__restrict__ sup) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)n_classes * nmem) return;
    int x = members[i];
    int *o = sup + i * 9;
    o[0] = x;
    float f;
    for (int mu = 0; mu < 4; ++mu) {
        o[1 + 2 * mu] = neighbour(g, x, mu, +1, &f);
        o[2 + 2 * mu] = neighbour(g, x, mu, -1, &f);
    }
}

int build_star_support(smpq_ctx *ctx, Buf &supsite, int *n_sup) {
    const int nsup = 9 * ctx->members;
    int rc = ensure(ctx, supsite, (size_t)ctx->n_classes * nsup * sizeof(int));
    if (rc) return rc;
    long n = (long)ctx->n_classes * ctx->members;
    star_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ctx->geom, (const int *)ctx->d_members.p,
                                                                      ctx->n_classes, ctx->members, (int *)supsite.p);
    *n_sup = nsup;
    return SMPQ_OK;
}

// y += c0 b on the support (y layout [j/BC][n_sup][12][BC]; supsite null: entry = site)
__global__ void add_c0b_kernel(int n_sup, int B, int BC, const int *__restrict__ supsite,
                               const int *__restrict__ rhs_class, const int *__restrict__ src_comp,
                               const int *__restrict__ colour, double c0, double2 *__restrict__ y) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)n_sup * B) return;
    int j = (int)(i % B), k = (int)(i / B);
    int cl = rhs_class[j];
    if (cl < 0) return;
    int site = supsite ? supsite[(size_t)cl * n_sup + k] : k;
    if (colour[site] != cl) return;
    int c = src_comp[j];
    size_t o = (((size_t)(j / BC) * n_sup + k) * 12 + c) * BC + (j % BC);
    y[o].x += c0;
}

void launch_add_c0b(int n_sup, int B, int BC, const int *d_supsite, const int *d_rhs_class, const int *d_src_comp,
                    const int *d_colour, double c0, double2 *y, cudaStream_t st) {
    long n = (long)n_sup * B;
    add_c0b_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_sup, B, BC, d_supsite, d_rhs_class, d_src_comp,
                                                                d_colour, c0, y);
}

// z = D_W y at member m of rhs j's class, from the star entries 9m..9m+8;
// qterm[(class * 12 + comp) * members + m] = gamma5(comp) z[comp] (Eqs. 5, 16).
template <int BC>
__global__ void contract_kernel(Geom g, const double2 *__restrict__ U, const double2 *__restrict__ y, int n_sup, int B,
                                const int *__restrict__ rhs_class, const int *__restrict__ src_comp,
                                const int *__restrict__ members, int nmem, double kappa, double2 *__restrict__ qterm) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)nmem * B) return;
    int j = (int)(i % B), m = (int)(i / B);
    int cl = rhs_class[j];
    if (cl < 0) return;
    int x = members[(size_t)cl * nmem + m];
    const double2 *yb = y + (size_t)(j / BC) * 12 * n_sup * BC + (j % BC);
    double2 acc[12][1];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c][0] = make_double2(0, 0);
    const int k0 = 9 * m;
    float f;
#define SMPQ_HOP(MU)                                                                                                   \
    {                                                                                                                  \
        neighbour(g, x, MU, +1, &f);                                                                                   \
        hop_one<double, MU, -1, false, BC>(U, yb, n_sup, g.V, k0 + 1 + 2 * MU, x, f < 0, acc);                        \
        int xb = neighbour(g, x, MU, -1, &f);                                                                          \
        hop_one<double, MU, +1, true, BC>(U, yb, n_sup, g.V, k0 + 2 + 2 * MU, xb, f < 0, acc);                        \
    }
    SMPQ_HOP(0)
    SMPQ_HOP(1)
    SMPQ_HOP(2)
    SMPQ_HOP(3)
#undef SMPQ_HOP
    int c = src_comp[j];
    double2 yc = yb[((size_t)k0 * 12 + c) * BC];
    double2 z = make_double2(yc.x - kappa * acc[c][0].x, yc.y - kappa * acc[c][0].y);
    double g5 = (c / 3) < 2 ? 1.0 : -1.0;
    qterm[((size_t)cl * 12 + c) * nmem + m] = make_double2(g5 * z.x, g5 * z.y);
}

void launch_contract(const Geom &g, const double *U64, const double2 *y, int n_sup, int B, int BC,
                     const int *d_rhs_class, const int *d_src_comp, const int *d_members, int members, double kappa,
                     double2 *qterm, cudaStream_t st) {
    long n = (long)members * B;
    unsigned grid = (unsigned)((n + 127) / 128);
    const double2 *U = (const double2 *)U64;
    switch (BC) {
    case 1: contract_kernel<1><<<grid, 128, 0, st>>>(g, U, y, n_sup, B, d_rhs_class, d_src_comp, d_members, members, kappa, qterm); break;
    case 12: contract_kernel<12><<<grid, 128, 0, st>>>(g, U, y, n_sup, B, d_rhs_class, d_src_comp, d_members, members, kappa, qterm); break;
    case 24: contract_kernel<24><<<grid, 128, 0, st>>>(g, U, y, n_sup, B, d_rhs_class, d_src_comp, d_members, members, kappa, qterm); break;
    case 48: contract_kernel<48><<<grid, 128, 0, st>>>(g, U, y, n_sup, B, d_rhs_class, d_src_comp, d_members, members, kappa, qterm); break;
    default: break;
    }
}

// Whole-lattice variant (the star-support ablation): z = D_W y is a field in
// the tile layout; qterm[(class * 12 + comp) * members + m] = gamma5(comp) z(x_m, comp, j).
__global__ void contract_full_kernel(const double2 *__restrict__ z, int V, int B, int BC,
                                     const int *__restrict__ rhs_class, const int *__restrict__ src_comp,
                                     const int *__restrict__ members, int nmem, double2 *__restrict__ qterm) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)nmem * B) return;
    int j = (int)(i % B), m = (int)(i / B);
    int cl = rhs_class[j];
    if (cl < 0) return;
    int x = members[(size_t)cl * nmem + m], c = src_comp[j];
    double2 v = z[(((size_t)(j / BC) * V + x) * 12 + c) * BC + (j % BC)];
    double g5 = (c / 3) < 2 ? 1.0 : -1.0;
    qterm[((size_t)cl * 12 + c) * nmem + m] = make_double2(g5 * v.x, g5 * v.y);
}

void launch_contract_full(const double2 *z, int V, int B, int BC, const int *d_rhs_class, const int *d_src_comp,
                          const int *d_members, int members, double2 *qterm, cudaStream_t st) {
    long n = (long)members * B;
    contract_full_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(z, V, B, BC, d_rhs_class, d_src_comp, d_members,
                                                                      members, qterm);
}

// q(x_m) = scale * sum_{comp = 0..11} qterm  (fixed order; scale 1/2 for Eq. 16)
__global__ void qsum_kernel(const double2 *__restrict__ qterm, const int *__restrict__ classes, int nc,
                            const int *__restrict__ members, int nmem, double *__restrict__ q_re,
                            double *__restrict__ q_im, double scale) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)nc * nmem) return;
    int cl = classes[i / nmem], m = (int)(i % nmem);
    double re = 0, im = 0;
    for (int c = 0; c < 12; ++c) {
        double2 v = qterm[((size_t)cl * 12 + c) * nmem + m];
        re += v.x;
        im += v.y;
    }
    int x = members[(size_t)cl * nmem + m];
    q_re[x] = scale * re;
    q_im[x] = scale * im;
}

void launch_qsum(const double2 *qterm, const int *d_classes, int nc, const int *d_members, int members, double *q_re,
                 double *q_im, double scale, cudaStream_t st) {
    long n = (long)nc * members;
    qsum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(qterm, d_classes, nc, d_members, members, q_re, q_im,
                                                             scale);
}

// ---------------------------------------------------------------- SMP trace of D_W^{-1} (Sec. 4 outlook)
__global__ void class_source_kernel(int V, int B, int BC, const int *__restrict__ colour,
                                    const int *__restrict__ rhs_class, const int *__restrict__ src_comp,
                                    double2 *__restrict__ b) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)V * 12 * B) return;
    int jj = (int)(i % BC);
    long r = i / BC;
    int c = (int)(r % 12);
    r /= 12;
    int s = (int)(r % V);
    int chunk = (int)(r / V);
    int j = chunk * BC + jj;
    int cl = rhs_class[j];
    b[i] = make_double2((cl >= 0 && colour[s] == cl && c == src_comp[j]) ? 1.0 : 0.0, 0.0);
}

void launch_class_source(int V, int B, int BC, const int *d_colour, const int *d_rhs_class, const int *d_src_comp,
                         double2 *b, cudaStream_t st) {
    long n = (long)V * 12 * B;
    class_source_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(V, B, BC, d_colour, d_rhs_class, d_src_comp, b);
}

__global__ void trace_terms_kernel(const double2 *__restrict__ y, int n_sup, int B, int BC,
                                   const int *__restrict__ rhs_class, const int *__restrict__ src_comp, int nmem,
                                   double2 *__restrict__ qterm) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)nmem * B) return;
    int j = (int)(i % B), m = (int)(i / B);
    int cl = rhs_class[j];
    if (cl < 0) return;
    int c = src_comp[j];
    // star entry 9 m is the member site itself
    double2 v = y[(((size_t)(j / BC) * n_sup + 9 * (size_t)m) * 12 + c) * BC + (j % BC)];
    qterm[((size_t)cl * 12 + c) * nmem + m] = v;
}

void launch_trace_terms(const double2 *y, int n_sup, int B, int BC, const int *d_rhs_class, const int *d_src_comp,
                        int members, double2 *qterm, cudaStream_t st) {
    long n = (long)members * B;
    trace_terms_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, n_sup, B, BC, d_rhs_class, d_src_comp, members,
                                                                    qterm);
}

// one block: out[0] = sum q_re (fixed order), out[1] = max |q_im|
__global__ void qtotal_kernel(const double *__restrict__ q_re, const double *__restrict__ q_im,
                              const int *__restrict__ sites, int n, double *out) {
    __shared__ double s_sum[1024], s_max[1024];
    double sum = 0, mx = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int x = sites ? sites[i] : i;
        sum += q_re[x];
        mx = fmax(mx, fabs(q_im[x]));
    }
    s_sum[threadIdx.x] = sum;
    s_max[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            s_sum[threadIdx.x] += s_sum[threadIdx.x + st];
            s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + st]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s_sum[0];
        out[1] = s_max[0];
    }
}

void launch_qtotal(const double *q_re, const double *q_im, const int *d_sites, int n, double *out2, cudaStream_t st) {
    qtotal_kernel<<<1, 1024, 0, st>>>(q_re, q_im, d_sites, n, out2);
}
