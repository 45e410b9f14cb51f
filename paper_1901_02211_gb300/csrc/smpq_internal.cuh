// Internal declarations of libsmpq (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <string>
#include <vector>

#include "../../include/smpq.h"
#include "df64.cuh"

#define SMPQ_MAX_POLES 32

// ---------------------------------------------------------------- complex helpers
template <typename T> struct cplx_t;
template <> struct cplx_t<double> { typedef double2 type; };
template <> struct cplx_t<float> { typedef float2 type; };
template <> struct cplx_t<df64> { typedef df64c type; };

// explicit conversion of a real component to double
__host__ __device__ __forceinline__ double to_d(double v) { return v; }
__host__ __device__ __forceinline__ double to_d(float v) { return v; }
__host__ __device__ __forceinline__ double to_d(df64 v) { return (double)v; }

template <typename C> __host__ __device__ __forceinline__ C mkc(double re, double im) {
    C c;
    c.x = re;
    c.y = im;
    return c;
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * b
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
    return acc;
}
// acc + conj(a) * b
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
    return acc;
}
__device__ __forceinline__ float2 cfmac(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
    return acc;
}
// i * a
__device__ __forceinline__ double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ double norm2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double norm2(float2 a) { return (double)a.x * a.x + (double)a.y * a.y; }

// ---------------------------------------------------------------- lattice geometry
struct Geom {
    int n[4];      // nx, ny, nz, nt
    int stride[4]; // 1, nx, nx*ny, nx*ny*nz
    int V;
    float bcf[4];  // boundary factor for hops crossing the boundary in mu
};

// Neighbour of s in direction mu (dir = +1 or -1); *f receives the boundary factor.
__device__ __forceinline__ int neighbour(const Geom &g, int s, int mu, int dir, float *f) {
    int c = (s / g.stride[mu]) % g.n[mu];
    if (dir > 0) {
        if (c == g.n[mu] - 1) {
            *f = g.bcf[mu];
            return s - (g.n[mu] - 1) * g.stride[mu];
        }
        *f = 1.f;
        return s + g.stride[mu];
    }
    if (c == 0) {
        *f = g.bcf[mu];
        return s + (g.n[mu] - 1) * g.stride[mu];
    }
    *f = 1.f;
    return s - g.stride[mu];
}

// ---------------------------------------------------------------- field layout
// A batch of B right-hand sides is stored in RHS tiles of BC columns:
//   element (component c in 0..11 = spin*3 + colour, site s, rhs j)
//   at (((j / BC) * V + s) * 12 + c) * BC + (j % BC),
// i.e. one tile is [site][component][column]: a warp reads consecutive columns
// of one site component, and the 12 components of a site sit at fixed
// offsets (immediates in the load instructions).
// Links: U[(mu * V + s) * 9 + row * 3 + col] (the 9 elements of one link contiguous).

// ---------------------------------------------------------------- solver state
struct ShiftParams {
    int n;                      // number of shifts
    double s0;                  // base shift (smallest q)
    double sig[SMPQ_MAX_POLES]; // q_i - s0
    double c[SMPQ_MAX_POLES];   // rational coefficients c_i
};

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct smpq_ctx {
    int device = 0;
    cudaStream_t stream = nullptr; // owned by the context
    void *user_stream = nullptr;   // caller's stream: its queued work precedes every call
    double last_Q = 0;
    smpq_options opt;
    std::string err;

    // lattice + links
    bool have_gauge = false;
    Geom geom;
    int dims[4] = {0, 0, 0, 0};
    int V = 0;
    Buf U64, U32, Udf; // FP64, FP32 and float-float copies of the links

    // spectrum / rational
    bool have_spec = false;
    double lmin2 = 0, lmax2 = 0, c0 = 0, delta = 0;
    std::vector<double> zc, zq;

    // colouring
    bool have_sources = false;
    int r = 0, mode = 0, n_classes = 0, members = 0; // members = sites per class
    std::vector<int> colour;                        // host copy [V]
    Buf d_colour;                                   // int[V]
    Buf d_members;                                  // int[n_classes][members] (site order)

    // workspace (grown on demand)
    std::vector<Buf> ws;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, evA = nullptr, evB = nullptr;
    // launch accounting and optional per-launch timing of the solver's D_W kernels
    long long launches = 0;
    // autotuned RHS tile width per (V, B, precision)
    std::vector<std::array<int, 4>> tuned; // {V, B, prec, BC}
    int last_bc = 0;
    std::vector<cudaEvent_t> prof_ev; // 4 per iteration of one check interval
    double prof_a_ms = 0, prof_b_ms = 0;         // FP32 iterations
    long long prof_a_n = 0, prof_b_n = 0;
    double prof_a_hi_ms = 0, prof_b_hi_ms = 0;   // FP64-accurate iterations
    long long prof_a_hi_n = 0, prof_b_hi_n = 0;
};

// workspace slots of smpq_ctx::ws
enum WsId {
    W_P, W_T, W_R, W_XLO, W_XHI, W_T64, W_PS, W_Y, W_PART, W_SCAL, W_B64,
    W_SRC, W_OUT, W_SUP, W_QTERM, W_RHS, W_Q, W_MISC, W_COUNT
};

// ---------------------------------------------------------------- host helpers
int set_err(smpq_ctx *ctx, int code, const std::string &msg);
int cuda_check(smpq_ctx *ctx, cudaError_t e, const char *what);
int ensure(smpq_ctx *ctx, Buf &b, size_t bytes);
void release(Buf &b);

// zolotarev.cpp
int zolotarev_coeffs(int n, double a, double b, double *c0, double *c, double *q, double *delta);
// host tridiagonal eigenvalue extremes (Sturm bisection)
void tridiag_extremes(const std::vector<double> &diag, const std::vector<double> &off, double *lo, double *hi);

// probing.cu (host part)
int colour_sites_host(const int dims[4], int r, int mode, std::vector<int> &colour, int *n_classes,
                      std::string *why);

// ---------------------------------------------------------------- kernel launchers
// dslash.cu
void launch_pack_links(const double *U_aos, double *U64, float *U32, void *Udf, int V, cudaStream_t st);
void launch_su3_check(const double *U64, int V, double *dev_maxerr, cudaStream_t st);
// convert ABI spinors [V][12][B] (FP64) <-> internal tiled layout of precision T
template <typename T> void launch_to_tiled(const double *in, void *out, int V, int B, int BC, cudaStream_t st);
template <typename T> void launch_from_tiled(const void *in, double *out, int V, int B, int BC, cudaStream_t st);
// out = D_W in (or D_W^dag), tiled layout, no reductions
template <typename T> void launch_dslash(const Geom &g, const void *U, const void *in, void *out, int B, int BC,
                                         int dagger, double kappa, cudaStream_t st);

// msolve.cu : multi-shift CG over a batch (see msolve.cu for the contract)
struct SolveSpec {
    int B, BC;                 // right-hand sides and tile width
    int prec;                  // SMPQ_FP64 / SMPQ_FP32 / SMPQ_MIXED
    int full_support;          // 1: shifted vectors on every site (apply_dov); 0: star support
    int n_sup;                 // support entries per rhs
    const int *d_supsite;      // [n_sup_classes][n_sup] site of support entry k for a class
    const int *d_rhs_class;    // [B] class (row of d_supsite) of rhs j, -1 for padding
    const int *d_colour;       // [V] class of each site (source definition)
    const int *d_src_class;    // [B] colour class whose sites carry rhs j's source (-1: none)
    const int *d_src_comp;     // [B] source component (spin*3 + colour) of rhs j
    const double *d_src_field; // optional explicit FP64 source in the solver's tiled layout
    const ShiftParams *shifts; // nullable: shifts and coefficients other than the context's rational
};
struct SolveOut {
    // y = R(H^2) b on the support, FP64, layout [(j/BC)*12 + c][n_sup][BC]
    double2 *y = nullptr;
    int iterations = 0;
    int reliable_updates = 0;
    double max_resid = 0;
    float solve_ms = 0;
};
int multishift_solve(smpq_ctx *ctx, const SolveSpec &spec, SolveOut *out);
int lanczos_extremes(smpq_ctx *ctx, int iters, double *lo, double *hi);
// autotuner: average ms of one D_W + D_W^dag-update launch pair (scratch fields in buf:
// 3 fields of B x 12 x V complex of the widest type used, part: partials, alpha: B doubles)
float time_dslash_pair(smpq_ctx *ctx, int prec, int B, int BC, int reps, void *buf, double *part, double *alpha);

// probing.cu : sources, star support, contraction, Q
int build_star_support(smpq_ctx *ctx, Buf &supsite, int *n_sup);
// y += c0 b on the star support of every rhs (b = 1 at component src_comp[j]
// of sites in class rhs_class[j])
void launch_add_c0b(int n_sup, int B, int BC, const int *d_supsite, const int *d_rhs_class, const int *d_src_comp,
                    const int *d_colour, double c0, double2 *y, cudaStream_t st);
// qterm[(class*12 + comp) * members + m] = gamma5_comp * (D_W y_j)(x_m)[comp] for
// every member m of rhs j's class (star support layout)
void launch_contract(const Geom &g, const double *U64, const double2 *y, int n_sup, int B, int BC,
                     const int *d_rhs_class, const int *d_src_comp, const int *d_members, int members, double kappa,
                     double2 *qterm, cudaStream_t st);
// q(x_m) = 1/2 sum_comp qterm for the listed classes
void launch_qsum(const double2 *qterm, const int *d_classes, int nc, const int *d_members, int members, double *q_re,
                 double *q_im, double scale, cudaStream_t st);
// tiled FP64 class sources: b_j(s, c) = 1 if colour[s] == rhs_class[j] and c == src_comp[j]
void launch_class_source(int V, int B, int BC, const int *d_colour, const int *d_rhs_class, const int *d_src_comp,
                         double2 *b, cudaStream_t st);
// qterm[(class * 12 + comp) * members + m] = y_j(member m)[comp] (diagonal of the solution, no gamma_5)
void launch_trace_terms(const double2 *y, int n_sup, int B, int BC, const int *d_rhs_class, const int *d_src_comp,
                        int members, double2 *qterm, cudaStream_t st);
// out[0] = sum of q_re over the listed sites (all when d_sites == nullptr), out[1] = max |q_im|
void launch_qtotal(const double *q_re, const double *q_im, const int *d_sites, int n, double *out2, cudaStream_t st);
