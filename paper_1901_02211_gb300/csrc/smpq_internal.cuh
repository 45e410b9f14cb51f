// Internal declarations of libsmpq (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <string>
#include <vector>

#include "../../include/smpq.h"
#include "device.cuh"

#define SMPQ_MAX_POLES 32

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
    Buf d_err;         // int: set by a staged D_W whose staging wait ran out
    Buf Uh16, Ub16;    // rows 0 and 1 of the links in FP16 and BF16 (reconstruct-12)

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
    // autotuned D_W launch shape per (lattice, B, precision): {BC, tiles per
    // block FP64-accurate / FP32, columns per thread}; from_file: read from the cache
    struct Tuned {
        std::array<int, 4> dims;
        int B, prec;
        std::array<int, 5> shape; // bc, tpb_hi, tpb_lo, nr, staged (bits: FP32, float-float)
        int from_file;
    };
    std::vector<Tuned> tuned;
    std::string tune_cache; // path of the tuning cache file ("" = none)
    int last_bc = 0;
    std::vector<cudaEvent_t> prof_ev; // 4 per iteration of one check interval
    double prof_a_ms = 0, prof_b_ms = 0;         // FP32 iterations
    long long prof_a_n = 0, prof_b_n = 0;
    double prof_a_hi_ms = 0, prof_b_hi_ms = 0;   // FP64-accurate iterations
    long long prof_a_hi_n = 0, prof_b_hi_n = 0;
    // low modes of H_W treated exactly (lowmodes.cu): lm_k > 0 switches the
    // projection on in compute_qx and apply_dov
    int lm_k = 0, lm_m = 0;     // modes in use, columns of the block
    Buf lm_vec;                 // FP64 tiled [m columns, tile 12], ordered by |lambda|
    Buf lm_sgn;                 // double[lm_k]: sign(lambda_j)
    Buf lm_w;                   // class overlaps v_j^dag b (per compute_qx call)
    std::vector<double> lm_val; // lambda_j, j < lm_m, ordered by |lambda|
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
// SMPQ_EINVAL unless p is device (or managed) memory of the context's GPU;
// `what` names the argument in the message
int check_device_ptr(smpq_ctx *ctx, const void *p, const char *what);

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

// half.cu : SMPQ_FP16N / SMPQ_BF16N storage for the stand-alone D_W.  A half
// field of B columns is one buffer of half_field_bytes(V, B): the components
// [j / BC][V][12][BC] (BC = half_tile(B)) followed by the norms [j / BC][V][BC].
void launch_pack_links12(const double *U_aos, void *Uh, void *Ub, int V, cudaStream_t st);
int half_tile(int B);
size_t half_field_bytes(int V, int B);
void launch_to_half(int prec, const double *in, void *out, int V, int B, cudaStream_t st);
void launch_from_half(int prec, const void *in, double *out, int V, int B, cudaStream_t st);
// the FP32 D_W with staged neighbour sites (stage.cuh), tiles of BC = 12, 24 or
// 48 columns; *err (device int, zero on entry) is set if a staging wait ran out
cudaError_t launch_dslash_staged(const Geom &g, const void *U, const void *in, void *out, int B, int BC, int dagger,
                                 double kappa, int *err, cudaStream_t st);
void launch_dslash_half(int prec, const Geom &g, const void *U, const void *in, void *out, int B, int dagger,
                        double kappa, cudaStream_t st);

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
    // shape of the D_W launches (the autotuner's choice; 0: 4, 4, 1): tiles per
    // block in the FP64-accurate and in the FP32 / half iterations, columns
    // per thread of the FP32 kernels (1 or 2)
    int tpb_hi, tpb_lo, nr;
    int staged; // D_W pair with neighbours staged in shared memory: bit 0 the FP32 iterations
                // (nr = 1), bit 1 the float-float iterations
};
struct SolveOut {
    // y = R(H^2) b on the support, FP64, layout [j/BC][n_sup][12][BC] (the field
    // tile layout when the support is the whole lattice)
    double2 *y = nullptr;
    int iterations = 0;
    int reliable_updates = 0;
    double max_resid = 0;
    double true_resid = -1; // max_j |b - (A + s0) x|/|b| of the base system (-1: not computed)
    float solve_ms = 0;
};
int multishift_solve(smpq_ctx *ctx, const SolveSpec &spec, SolveOut *out);
// one solve over n (1..4) lattices of different sizes, their right-hand sides
// in the same launches (ctxs[0] supplies stream, workspace and options; every
// spec has the same precision and tile width and its own B, support, sources)
int multishift_solve_batch(smpq_ctx *const *ctxs, const SolveSpec *specs, SolveOut *outs, int n);
int lanczos_extremes(smpq_ctx *ctx, int iters, double *lo, double *hi);
// lowmodes.cu : the k + 1 eigenpairs of H_W of smallest |lambda| (block of m
// columns, m a multiple of 12, at most 48) into ctx->lm_*; evals / resid get
// k + 1 entries
int lowmodes_compute(smpq_ctx *ctx, int k, int m, double tol, int max_iter, int degree, double *evals,
                     double *resid, int *iterations);
void lowmodes_clear(smpq_ctx *ctx);
// projection of the SMP sources of one batch: w = v^dag b per class (once per
// call, for classes listed in d_classes), b_perp = b - V w into the tiled
// source field, y += c0 b_perp on the support, and the low-mode term of q(x)
int lowmodes_class_overlaps(smpq_ctx *ctx, cudaStream_t st);
void lowmodes_source(smpq_ctx *ctx, double2 *bperp, int B, int BC, const int *d_rhs_class, const int *d_src_comp,
                     cudaStream_t st);
void lowmodes_add_c0b(smpq_ctx *ctx, int n_sup, int B, int BC, const int *d_supsite, const int *d_rhs_class,
                      const double2 *bperp, double2 *y, cudaStream_t st);
void lowmodes_qterm(smpq_ctx *ctx, const int *d_classes, int nc, double2 *qterm, cudaStream_t st);
// apply_dov (tile 1, B columns): b_perp = b - V (V^dag b) into bperp, keeping
// V^dag b for lowmodes_dov_finish, which adds gamma_5 V sign (V^dag b) to out
int lowmodes_dov_project(smpq_ctx *ctx, const double2 *b, double2 *bperp, int B, std::vector<double> &wd,
                         cudaStream_t st);
int lowmodes_dov_finish(smpq_ctx *ctx, double2 *out, int B, const std::vector<double> &wd, cudaStream_t st);
// autotuner: average ms of one D_W + D_W^dag-update launch pair of the
// iterations of `kind` (0 FP64, 1 FP32, 2 float-float, 3 FP16 + norms,
// 4 BF16 + norms, 5 FP32 with staged neighbours, 6 float-float with staged
// neighbours) for B columns in tiles of BC,
// tpb tiles per block and nr columns per thread (FP32: 1 or 2).  Scratch in
// buf: 3 fields of B x 12 x V complex values of the kind; part: 2 * B * V / 12
// doubles of partials; alpha: B doubles; err: one int, zero on entry (kind 5
// sets it if a staging wait ran out).  -1 on a bad shape or a CUDA error.
float time_dslash_pair(smpq_ctx *ctx, int kind, int B, int BC, int tpb, int nr, int reps, void *buf, double *part,
                       double *alpha, int *err);

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
// the same from z = D_W y on the whole lattice (field tile layout), for the
// full-support ablation
void launch_contract_full(const double2 *z, int V, int B, int BC, const int *d_rhs_class, const int *d_src_comp,
                          const int *d_members, int members, double2 *qterm, cudaStream_t st);
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
