// C ABI of libsmpq (declared and documented in include/smpq.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "smpq_internal.cuh"

// ------------------------------------------------------------------ helpers
int set_err(smpq_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_check(smpq_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SMPQ_OK;
    return set_err(ctx, e == cudaErrorMemoryAllocation ? SMPQ_ENOMEM : SMPQ_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

int ensure(smpq_ctx *ctx, Buf &b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return SMPQ_OK;
    release(b);
    if (bytes == 0) return SMPQ_OK;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        b.bytes = 0;
        return set_err(ctx, SMPQ_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    b.bytes = bytes;
    return SMPQ_OK;
}

void release(Buf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

int check_device_ptr(smpq_ctx *ctx, const void *p, const char *what) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, SMPQ_EINVAL, std::string(what) + ": not a pointer CUDA knows");
    }
    if (a.type == cudaMemoryTypeManaged) return SMPQ_OK;
    if (a.type != cudaMemoryTypeDevice)
        return set_err(ctx, SMPQ_EINVAL, std::string(what) + ": a device buffer was expected, got host memory");
    if (a.device != ctx->device)
        return set_err(ctx, SMPQ_EINVAL, std::string(what) + ": device memory of GPU " + std::to_string(a.device) +
                                             ", the context runs on GPU " + std::to_string(ctx->device));
    return SMPQ_OK;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// make the context stream wait for work already queued on the caller's stream
struct StreamEntry {
    StreamEntry(smpq_ctx *ctx, void *user) {
        if (user) {
            cudaEventRecord(ctx->ev0, (cudaStream_t)user);
            cudaStreamWaitEvent(ctx->stream, ctx->ev0, 0);
        }
    }
};

__global__ void k_axpy(double2 *__restrict__ y, const double2 *__restrict__ x, double a, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) {
        y[i].x += a * x[i].x;
        y[i].y += a * x[i].y;
    }
}

void launch_axpy(double2 *y, const double2 *x, double a, size_t n, cudaStream_t st) {
    k_axpy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, x, a, n);
}

int check_ctx(smpq_ctx *ctx, bool gauge, bool spec, bool src) {
    if (!ctx) return SMPQ_EINVAL;
    if (gauge && !ctx->have_gauge) return set_err(ctx, SMPQ_ESTATE, "no gauge field loaded");
    if (spec && !ctx->have_spec) return set_err(ctx, SMPQ_ESTATE, "no spectrum interval set");
    if (src && !ctx->have_sources) return set_err(ctx, SMPQ_ESTATE, "no colouring scheme built");
    return SMPQ_OK;
}

int validate_options(smpq_ctx *ctx, const smpq_options *o) {
    if (!(o->kappa > 0) || !(o->kappa < 1)) return set_err(ctx, SMPQ_EINVAL, "kappa must be in (0, 1)");
    if (o->npoles < 1 || o->npoles > SMPQ_MAX_POLES) return set_err(ctx, SMPQ_EINVAL, "npoles must be in 1..32");
    if (!(o->tol > 0) || !(o->tol < 1)) return set_err(ctx, SMPQ_EINVAL, "tol must be in (0, 1)");
    if (o->max_iter < 1) return set_err(ctx, SMPQ_EINVAL, "max_iter must be positive");
    if (o->precision != SMPQ_FP64 && o->precision != SMPQ_FP32 && o->precision != SMPQ_MIXED &&
        o->precision != SMPQ_FP16N && o->precision != SMPQ_BF16N)
        return set_err(ctx, SMPQ_EINVAL, "bad precision");
    if (o->precision == SMPQ_MIXED && (!(o->switch_residual > 0) || !(o->switch_residual < 1)))
        return set_err(ctx, SMPQ_EINVAL, "switch_residual must be in (0, 1)");
    if (!(o->reliable_delta > 0) || !(o->reliable_delta < 1))
        return set_err(ctx, SMPQ_EINVAL, "reliable_delta must be in (0, 1)");
    for (int mu = 0; mu < 4; ++mu)
        if (o->bc[mu] != 1 && o->bc[mu] != -1) return set_err(ctx, SMPQ_EINVAL, "bc must be +1 or -1");
    if (o->rhs_block < 0 || (o->rhs_block > 1 && o->rhs_block % 12))
        return set_err(ctx, SMPQ_EINVAL, "rhs_block must be 0, 1 or a multiple of 12");
    if (o->iters_per_check < 1) return set_err(ctx, SMPQ_EINVAL, "iters_per_check must be positive");
    if (o->staging < -1 || o->staging > 1) return set_err(ctx, SMPQ_EINVAL, "staging must be -1, 0 or 1");
    return SMPQ_OK;
}

void set_geom(smpq_ctx *ctx) {
    Geom &g = ctx->geom;
    int st = 1;
    for (int mu = 0; mu < 4; ++mu) {
        g.n[mu] = ctx->dims[mu];
        g.stride[mu] = st;
        st *= ctx->dims[mu];
        g.bcf[mu] = (float)ctx->opt.bc[mu];
    }
    g.V = ctx->V;
}

// ---------------------------------------------------------------- autotuner
// The shape of the solver's D_W launches: RHS tile width BC (12, 24 or 48,
// shared by both phases of the mixed solve: its fields change precision in
// place), tiles per block of the FP64-accurate and of the FP32 / half-storage
// iterations (1, 2, 4 or 8), and columns per thread of the FP32 kernels (1 or
// 2).  Chosen once per (device, lattice, B, precision) by timing the D_W pair
// of every candidate on the solver's own workspace; kept in the context and,
// with opt.tune_cache set, in a text file that later processes read first.
struct Shape {
    int bc, tpb_hi, tpb_lo, nr, staged;
};
constexpr int TPB_DEFAULT = 4;    // tiles per block of the FP32 / half / FP64 D_W launches (msolve.cu)
constexpr int TPB_DEFAULT_HI = 2; // of the float-float ones (the tuner's usual choice on a GB300)

std::string device_key(int dev) {
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    return std::string(pr.name) + "/" + std::to_string(pr.multiProcessorCount) + "sm";
}

std::string cache_key(const char *device, const int dims[4], int B, int precision) {
    return std::string("smpq-tune-2|") + device + "|" + std::to_string(dims[0]) + " " + std::to_string(dims[1]) +
           " " + std::to_string(dims[2]) + " " + std::to_string(dims[3]) + "|" + std::to_string(B) + "|" +
           std::to_string(precision) + "|";
}

int tune_kind_lo(int prec) {
    return prec == SMPQ_FP64 ? 0 : prec == SMPQ_FP16N ? 3 : prec == SMPQ_BF16N ? 4 : 1;
}

Shape tune_shape_raw(smpq_ctx *ctx, int B, int prec, int *cached) {
    *cached = 0;
    Shape def{1, prec == SMPQ_MIXED ? TPB_DEFAULT_HI : TPB_DEFAULT, TPB_DEFAULT, 1, 0};
    if (B == 1) return def;
    std::vector<int> cand;
    for (int bc : {12, 24, 48})
        if (B % bc == 0) cand.push_back(bc);
    if (cand.empty()) return def;
    def.bc = cand.back();
    const int kind_lo = tune_kind_lo(prec);
    // staged neighbours (staging 1): bit 0 the FP32 iterations, bit 1 the float-float ones
    def.staged = ctx->opt.staging == 1 ? (kind_lo == 1 ? 1 : 0) | (prec == SMPQ_MIXED ? 2 : 0) : 0;
    if (!ctx->opt.autotune) return def;
    for (auto &e : ctx->tuned)
        if (e.dims == std::array<int, 4>{ctx->dims[0], ctx->dims[1], ctx->dims[2], ctx->dims[3]} && e.B == B &&
            e.prec == prec) {
            *cached = e.from_file;
            return Shape{e.shape[0], e.shape[1], e.shape[2], e.shape[3], e.shape[4]};
        }
    const std::string dev = device_key(ctx->device);
    int sh[5];
    if (!ctx->tune_cache.empty() &&
        smpq_tune_cache_lookup(ctx->tune_cache.c_str(), dev.c_str(), ctx->dims, B, prec, sh) == SMPQ_OK &&
        B % sh[0] == 0) {
        ctx->tuned.push_back({{ctx->dims[0], ctx->dims[1], ctx->dims[2], ctx->dims[3]}, B, prec, {sh[0], sh[1], sh[2], sh[3], sh[4]}, 1});
        *cached = 1;
        return Shape{sh[0], sh[1], sh[2], sh[3], sh[4]};
    }
    // scratch for the timing launches: three fields of the widest kind timed
    // (float-float or FP64: 16 bytes per complex value; FP32: 8; half storage:
    // p and t in the half format and r in FP32)
    const size_t nf = (size_t)B * 12 * ctx->V;
    const bool half = prec == SMPQ_FP16N || prec == SMPQ_BF16N;
    const size_t hb = ((nf * 4 + nf / 12 * 4) + 255) / 256 * 256;
    const size_t scratch = half ? 2 * hb + nf * sizeof(float2) : 3 * nf * (prec == SMPQ_FP32 ? sizeof(float2) : sizeof(df64c));
    if (ensure(ctx, ctx->ws[W_P], scratch) ||
        ensure(ctx, ctx->ws[W_PART], (size_t)2 * nf / 12 * sizeof(double) + 64) ||
        ensure(ctx, ctx->ws[W_SCAL], (size_t)B * sizeof(double) + 16)) {
        cudaGetLastError();
        return def;
    }
    cudaMemsetAsync(ctx->ws[W_P].p, 0, scratch, ctx->stream);
    cudaMemsetAsync(ctx->ws[W_SCAL].p, 0, (size_t)B * sizeof(double) + 16, ctx->stream);
    void *buf = ctx->ws[W_P].p;
    double *part = (double *)ctx->ws[W_PART].p, *alpha = (double *)ctx->ws[W_SCAL].p;
    int *err = (int *)(alpha + B); // staging-wait flag of the staged timings
    const bool mixed = prec == SMPQ_MIXED, fp64 = prec == SMPQ_FP64;
    Shape best = def;
    float tbest = 1e30f;
    for (int bc : cand) {
        Shape s{bc, 4, 4, 1, 0};
        float tlo = 1e30f, thi = 0.f;
        // the FP32 / half / FP64 iterations (FP64 runs with the tiles-per-block
        // of the FP64-accurate iterations); FP32 also with staged neighbours
        for (int tpb : {1, 2, 4, 8})
            for (int v : {0, 1, 2}) { // 0, 1: one or two columns per thread; 2: staged
                if (v > 0 && kind_lo != 1) continue;
                if (kind_lo == 1 && ((v == 2 && ctx->opt.staging == 0) || (v < 2 && ctx->opt.staging == 1)))
                    continue;
                const int nr = v == 1 ? 2 : 1;
                const float t = time_dslash_pair(ctx, v == 2 ? 5 : kind_lo, B, bc, tpb, nr, fp64 ? 2 : 3, buf, part,
                                                 alpha, err);
                ctx->launches += 2 * (1 + (fp64 ? 2 : 3));
                if (t > 0 && t < tlo) {
                    tlo = t;
                    if (fp64) s.tpb_hi = tpb;
                    else s.tpb_lo = tpb;
                    s.nr = nr;
                    s.staged = (s.staged & 2) | (v == 2 ? 1 : 0);
                }
            }
        if (mixed) { // the float-float iterations: about a quarter of the solve
            float th = 1e30f;
            for (int tpb : {1, 2, 4, 8})
                for (int v : {0, 1}) { // plain loads, staged neighbours
                    if ((v == 1 && ctx->opt.staging == 0) || (v == 0 && ctx->opt.staging == 1)) continue;
                    const float t = time_dslash_pair(ctx, v ? 6 : 2, B, bc, tpb, 1, 2, buf, part, alpha, err);
                    ctx->launches += 6;
                    if (t > 0 && t < th) {
                        th = t;
                        s.tpb_hi = tpb;
                        s.staged = (s.staged & 1) | (v ? 2 : 0);
                    }
                }
            thi = th;
        }
        const float est = mixed ? 0.25f * thi + 0.75f * tlo : tlo;
        if (est < tbest) {
            tbest = est;
            best = s;
        }
    }
    cudaGetLastError();
    ctx->tuned.push_back({{ctx->dims[0], ctx->dims[1], ctx->dims[2], ctx->dims[3]}, B, prec,
                          {best.bc, best.tpb_hi, best.tpb_lo, best.nr, best.staged}, 0});
    if (!ctx->tune_cache.empty()) {
        const int shape[5] = {best.bc, best.tpb_hi, best.tpb_lo, best.nr, best.staged};
        smpq_tune_cache_store(ctx->tune_cache.c_str(), dev.c_str(), ctx->dims, B, prec, shape, tbest);
    }
    return best;
}

// the tuned (or cached, or default) shape with the staging option applied
Shape tune_shape(smpq_ctx *ctx, int B, int prec, int *cached) {
    Shape s = tune_shape_raw(ctx, B, prec, cached);
    const int can = (tune_kind_lo(prec) == 1 ? 1 : 0) | (prec == SMPQ_MIXED ? 2 : 0); // stageable phases
    if (s.bc < 12 || ctx->opt.staging == 0) {
        s.staged = 0;
    } else if (ctx->opt.staging == 1) {
        s.staged = can;
        if (can & 1) s.nr = 1;
    } else {
        s.staged &= can;
    }
    return s;
}

// device bytes one right-hand side costs in the solver (full-lattice vectors)
size_t bytes_per_rhs(const smpq_ctx *ctx, int prec, int n_sup, int npoles) {
    const bool half = prec == SMPQ_FP16N || prec == SMPQ_BF16N;
    size_t per = prec == SMPQ_FP32 ? (4 * 8 + 2 * 16)
                 : half            ? (2 * 5 + 2 * 8 + 2 * 16) // p, t: 4 B + a 12th of the 4-byte norm
                                   : (prec == SMPQ_MIXED ? 4 * 16 + 4 * 8 : 3 * 16); // MIXED: p t r x_hi, p t r x_lo
    if (ctx->opt.true_residual && prec == SMPQ_FP64) per += 2 * 16; // x64, t64
    size_t full = (size_t)ctx->V * 12 * per;
    size_t eb = (prec == SMPQ_FP32 || half) ? 8 : (prec == SMPQ_MIXED ? 16 + 8 : 16); // MIXED: FP64 and FP32 copies
    size_t sup = (size_t)n_sup * 12 * (npoles * eb + 16);
    return full + sup;
}

// kind 0: q^SMP(x) of Eq. 16; kind 1: SMP estimate of diag D_W^{-1}
int compute_classes(smpq_ctx *ctx, const std::vector<int> &classes, double *q_re, double *q_im, int on_device,
                    smpq_stats *stats, bool full, int kind = 0) {
    cudaStream_t st = ctx->stream;
    if (on_device) {
        int rc0;
        if ((rc0 = check_device_ptr(ctx, q_re, "output (real parts)")) || (rc0 = check_device_ptr(ctx, q_im, "output (imaginary parts)")))
            return rc0;
    }
    ctx->launches = 0;
    ctx->prof_a_ms = ctx->prof_b_ms = ctx->prof_a_hi_ms = ctx->prof_b_hi_ms = 0;
    ctx->prof_a_n = ctx->prof_b_n = ctx->prof_a_hi_n = ctx->prof_b_hi_n = 0;
    cudaEventRecord(ctx->evA, st);
    int rc;
    // star support of every class
    int n_sup = 0;
    if ((rc = build_star_support(ctx, ctx->ws[W_SUP], &n_sup))) return rc;
    // ablation of the star support: shifted directions on every site
    const bool full_sup = kind == 0 && ctx->opt.full_support;
    if (full_sup) n_sup = ctx->V;
    const int prec = ctx->opt.precision;
    const int nc = (int)classes.size();
    const int nrhs_total = 12 * nc;
    // batch size
    int B;
    if (ctx->opt.rhs_block == 1) B = 1;
    else if (ctx->opt.rhs_block > 1) B = std::min(ctx->opt.rhs_block, nrhs_total);
    else {
        size_t freeb = 0, totb = 0;
        cudaMemGetInfo(&freeb, &totb);
        // the context's own workspace is reusable: count it as available, so
        // the batch size does not shrink from one call to the next
        size_t held = 0;
        for (const Buf &b : ctx->ws) held += b.bytes;
        size_t per = bytes_per_rhs(ctx, prec, n_sup, ctx->opt.npoles);
        if (kind == 0 && ctx->lm_k > 0) per += (size_t)ctx->V * 12 * sizeof(double2); // projected source field
        long cap = (long)((0.6 * (double)(freeb + held)) / (double)per);
        cap = std::max(12L, cap - cap % 48);
        B = (int)std::min<long>(nrhs_total, cap);
        if (B > 48) B -= B % 48;
    }
    if (B > 1) B -= B % 12;
    if (B < 1) B = 1;
    int from_cache = 0;
    const Shape shape = tune_shape(ctx, B, prec, &from_cache);
    const int BC = shape.bc;
    ctx->last_bc = BC;
    // qterm + device q
    if ((rc = ensure(ctx, ctx->ws[W_QTERM], (size_t)ctx->n_classes * 12 * ctx->members * sizeof(double2)))) return rc;
    if ((rc = ensure(ctx, ctx->ws[W_RHS], (size_t)3 * B * sizeof(int) + (size_t)nc * sizeof(int) +
                                           (size_t)nc * ctx->members * sizeof(int) + 4 * sizeof(double))))
        return rc;
    int *d_rhs_class = (int *)ctx->ws[W_RHS].p, *d_src_comp = d_rhs_class + B, *d_src_class = d_src_comp + B;
    int *d_classes = d_src_class + B, *d_sites = d_classes + nc;
    double *d_tot = (double *)(((uintptr_t)(d_sites + (size_t)nc * ctx->members) + 15) & ~(uintptr_t)15);
    std::vector<int> h_rhs(3 * (size_t)B);

    SolveSpec spec{};
    spec.B = B;
    spec.BC = BC;
    spec.prec = prec;
    spec.full_support = 0;
    spec.n_sup = n_sup;
    spec.d_supsite = full_sup ? nullptr : (const int *)ctx->ws[W_SUP].p;
    spec.full_support = full_sup ? 1 : 0;
    spec.d_rhs_class = d_rhs_class;
    spec.d_colour = (const int *)ctx->d_colour.p;
    spec.d_src_class = d_src_class;
    spec.d_src_comp = d_src_comp;
    spec.d_src_field = nullptr;
    spec.shifts = nullptr;
    spec.tpb_hi = shape.tpb_hi;
    spec.tpb_lo = shape.tpb_lo;
    spec.nr = shape.nr;
    spec.staged = shape.staged;
    ShiftParams cg; // kind 1: one unshifted system D_W^dag D_W x = D_W^dag b, y = x
    if (kind == 1) {
        cg.n = 1;
        cg.s0 = 0;
        cg.sig[0] = 0;
        cg.c[0] = 1;
        spec.shifts = &cg;
        const size_t nf = (size_t)ctx->V * 12 * B;
        if ((rc = ensure(ctx, ctx->ws[W_SRC], 2 * nf * sizeof(double2)))) return rc;
        spec.d_src_field = (const double *)((double2 *)ctx->ws[W_SRC].p + nf);
    }
    const bool project = kind == 0 && ctx->lm_k > 0; // low modes of H_W treated exactly
    if (project) {
        if ((rc = ensure(ctx, ctx->ws[W_SRC], (size_t)ctx->V * 12 * B * sizeof(double2)))) return rc;
        spec.d_src_field = (const double *)ctx->ws[W_SRC].p;
        if ((rc = lowmodes_class_overlaps(ctx, st))) return rc;
    }

    int maxit = 0, nrel = 0, nb = 0;
    long long totit = 0;
    double worst = 0, solve_ms = 0, true_res = -1;
    for (int j0 = 0; j0 < nrhs_total; j0 += B) {
        for (int j = 0; j < B; ++j) {
            int g = j0 + j;
            int cl = g < nrhs_total ? classes[g / 12] : -1;
            h_rhs[j] = cl;
            h_rhs[B + j] = g % 12;
            h_rhs[2 * B + j] = cl;
        }
        cudaMemcpyAsync(d_rhs_class, h_rhs.data(), 3 * (size_t)B * sizeof(int), cudaMemcpyHostToDevice, st);
        if (kind == 1) { // source D_W^dag b of the normal equations
            double2 *b = (double2 *)ctx->ws[W_SRC].p;
            launch_class_source(ctx->V, B, BC, spec.d_colour, d_rhs_class, d_src_comp, b, st);
            launch_dslash<double>(ctx->geom, ctx->U64.p, b, (void *)spec.d_src_field, B, BC, 1, ctx->opt.kappa, st);
            ctx->launches += 2;
        }
        if (project) lowmodes_source(ctx, (double2 *)ctx->ws[W_SRC].p, B, BC, d_rhs_class, d_src_comp, st);
        SolveOut out;
        rc = multishift_solve(ctx, spec, &out);
        if (rc) return rc;
        if (kind == 0) {
            if (project)
                lowmodes_add_c0b(ctx, n_sup, B, BC, spec.d_supsite, d_rhs_class, (const double2 *)ctx->ws[W_SRC].p,
                                 out.y, st);
            else
                launch_add_c0b(n_sup, B, BC, spec.d_supsite, d_rhs_class, d_src_comp, spec.d_colour, ctx->c0, out.y,
                               st);
            if (full_sup) { // y is a whole-lattice field: z = D_W y everywhere, read at the members
                if ((rc = ensure(ctx, ctx->ws[W_OUT], (size_t)ctx->V * 12 * B * sizeof(double2)))) return rc;
                double2 *z = (double2 *)ctx->ws[W_OUT].p;
                launch_dslash<double>(ctx->geom, ctx->U64.p, out.y, z, B, BC, 0, ctx->opt.kappa, st);
                launch_contract_full(z, ctx->V, B, BC, d_rhs_class, d_src_comp, (const int *)ctx->d_members.p,
                                     ctx->members, (double2 *)ctx->ws[W_QTERM].p, st);
                ctx->launches += 1;
            } else {
                launch_contract(ctx->geom, (const double *)ctx->U64.p, out.y, n_sup, B, BC, d_rhs_class,
                                d_src_comp, (const int *)ctx->d_members.p, ctx->members, ctx->opt.kappa,
                                (double2 *)ctx->ws[W_QTERM].p, st);
            }
        } else {
            launch_trace_terms(out.y, n_sup, B, BC, d_rhs_class, d_src_comp, ctx->members,
                               (double2 *)ctx->ws[W_QTERM].p, st);
        }
        ctx->launches += 2;
        maxit = std::max(maxit, out.iterations);
        totit += out.iterations;
        nrel += out.reliable_updates;
        worst = std::max(worst, out.max_resid);
        if (out.true_resid >= 0) true_res = std::max(true_res, out.true_resid);
        solve_ms += out.solve_ms;
        ++nb;
    }
    // q(x) of the processed classes
    cudaMemcpyAsync(d_classes, classes.data(), nc * sizeof(int), cudaMemcpyHostToDevice, st);
    double *dq_re, *dq_im;
    if (on_device) {
        dq_re = q_re;
        dq_im = q_im;
    } else {
        if ((rc = ensure(ctx, ctx->ws[W_Q], 2 * (size_t)ctx->V * sizeof(double)))) return rc;
        dq_re = (double *)ctx->ws[W_Q].p;
        dq_im = dq_re + ctx->V;
    }
    if (project) lowmodes_qterm(ctx, d_classes, nc, (double2 *)ctx->ws[W_QTERM].p, st);
    launch_qsum((const double2 *)ctx->ws[W_QTERM].p, d_classes, nc, (const int *)ctx->d_members.p, ctx->members,
                dq_re, dq_im, kind == 0 ? 0.5 : 1.0, st);
    // Q in site order over the processed sites
    std::vector<int> sites;
    if (!full) {
        sites.reserve((size_t)nc * ctx->members);
        std::vector<char> mark(ctx->n_classes, 0);
        for (int c : classes) mark[c] = 1;
        for (int s = 0; s < ctx->V; ++s)
            if (mark[ctx->colour[s]]) sites.push_back(s);
        cudaMemcpyAsync(d_sites, sites.data(), sites.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    }
    launch_qtotal(dq_re, dq_im, full ? nullptr : d_sites, full ? ctx->V : (int)sites.size(), d_tot, st);
    ctx->launches += 3 + 1; // qsum, qtotal, star support (+1)
    double tot[2];
    cudaMemcpyAsync(tot, d_tot, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (!on_device) {
        std::vector<double> hq(2 * (size_t)ctx->V);
        cudaMemcpyAsync(hq.data(), dq_re, hq.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_check(ctx, e, "compute_qx copy-out");
        if (full) {
            std::memcpy(q_re, hq.data(), ctx->V * sizeof(double));
            std::memcpy(q_im, hq.data() + ctx->V, ctx->V * sizeof(double));
        } else {
            for (int s : sites) {
                q_re[s] = hq[s];
                q_im[s] = hq[ctx->V + s];
            }
        }
    }
    cudaEventRecord(ctx->evB, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "compute_qx");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(ctx, e, "compute_qx launch");
    float tms = 0;
    cudaEventElapsedTime(&tms, ctx->evA, ctx->evB);
    if (stats) {
        stats->n_rhs = nrhs_total;
        stats->n_classes = nc;
        stats->n_batches = nb;
        stats->max_iterations = maxit;
        stats->total_iterations = totit;
        stats->reliable_updates = nrel;
        stats->max_resid = worst;
        stats->max_im_q = tot[1];
        stats->Q = tot[0];
        stats->q_round_dev = std::fabs(tot[0] - std::nearbyint(tot[0]));
        stats->true_resid = true_res;
        stats->tiles_per_block_hi = shape.tpb_hi;
        stats->tiles_per_block_lo = shape.tpb_lo;
        stats->cols_per_thread = shape.nr;
        stats->shape_from_cache = from_cache;
        stats->staged = BC > 1 ? shape.staged : 0;
        stats->solve_ms = solve_ms;
        stats->total_ms = tms;
        stats->kernel_launches = ctx->launches;
        stats->dslash_ms = ctx->prof_a_ms;
        stats->dslash_launches = ctx->prof_a_n;
        stats->update_ms = ctx->prof_b_ms;
        stats->update_launches = ctx->prof_b_n;
        stats->rhs_tile = ctx->last_bc;
        stats->dslash_hi_ms = ctx->prof_a_hi_ms;
        stats->dslash_hi_launches = ctx->prof_a_hi_n;
        stats->update_hi_ms = ctx->prof_b_hi_ms;
        stats->update_hi_launches = ctx->prof_b_hi_n;
    }
    ctx->last_Q = tot[0];
    return SMPQ_OK;
}

// The uneven batch: q^SMP(x) on n lattices of different sizes (1 <= n <= 4,
// one context each), their right-hand sides solved together: every CG
// iteration is the same three launches for all lattices (each RHS tile knows
// its lattice's geometry, links and rational).  The sources run in rounds;
// each round takes about the same share of every lattice's sources, so all
// rounds mix the lattices, and the rounds fit the device memory the first
// context can use.
int compute_batch(smpq_ctx **ctxs, int n, double **q_re, double **q_im, int on_device, double *Q, smpq_stats *stats) {
    smpq_ctx *c0 = ctxs[0];
    cudaStream_t st = c0->stream;
    const int prec = c0->opt.precision;
    int rc;
    for (int l = 0; l < n; ++l) {
        smpq_ctx *c = ctxs[l];
        if ((rc = check_ctx(c, true, true, true))) return rc;
        if (c->device != c0->device || c->opt.precision != prec || c->opt.npoles != c0->opt.npoles)
            return set_err(c0, SMPQ_EINVAL, "uneven batch: every context needs the same device, precision and poles");
        if (c->lm_k > 0 || c->opt.full_support || c->opt.rhs_block == 1)
            return set_err(c0, SMPQ_EINVAL, "uneven batch: no low-mode projection, full support or one-rhs batches");
        if (on_device && ((rc = check_device_ptr(c0, q_re[l], "q_re")) || (rc = check_device_ptr(c0, q_im[l], "q_im"))))
            return rc;
        c->launches = 0;
        c->prof_a_ms = c->prof_b_ms = c->prof_a_hi_ms = c->prof_b_hi_ms = 0;
        c->prof_a_n = c->prof_b_n = c->prof_a_hi_n = c->prof_b_hi_n = 0;
    }
    cudaEventRecord(c0->evA, st);
    // every lattice's star support, qterm and class list
    std::vector<int> nsup(n), N(n);
    size_t need = 0, held = 0;
    for (int l = 0; l < n; ++l) {
        smpq_ctx *c = ctxs[l];
        if ((rc = build_star_support(c, c->ws[W_SUP], &nsup[l]))) return rc;
        if ((rc = ensure(c, c->ws[W_QTERM], (size_t)c->n_classes * 12 * c->members * sizeof(double2)))) return rc;
        N[l] = 12 * c->n_classes;
        need += (size_t)N[l] * bytes_per_rhs(c, prec, nsup[l], c->opt.npoles);
    }
    for (const Buf &b : c0->ws) held += b.bytes;
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    const double budget = 0.6 * (double)(freeb + held);
    int rounds = std::max(1, (int)std::ceil((double)need / budget));
    // per-round batch of each lattice: its share, rounded up to the tile
    // width (a small lattice pads its last round with empty columns, or ends
    // early); tiles of 12 only when every lattice has fewer than 48 sources
    int BC = 12;
    for (int l = 0; l < n; ++l)
        if (N[l] >= 48) BC = 48;
    std::vector<int> Bl(n);
    for (int l = 0; l < n; ++l) Bl[l] = ((N[l] + rounds - 1) / rounds + BC - 1) / BC * BC;
    rounds = 0;
    for (int l = 0; l < n; ++l) rounds = std::max(rounds, (N[l] + Bl[l] - 1) / Bl[l]);
    int Btot = 0;
    for (int l = 0; l < n; ++l) Btot += Bl[l];
    // launch shape: the default tiles per block, one column per thread (timing
    // candidates would need scratch the size of the round again)
    const int from_cache = 0;
    const Shape shape{BC, prec == SMPQ_MIXED ? TPB_DEFAULT_HI : TPB_DEFAULT, TPB_DEFAULT, 1,
                      c0->opt.staging == 1 ? (tune_kind_lo(prec) == 1 ? 1 : 0) | (prec == SMPQ_MIXED ? 2 : 0) : 0};
    // global per-rhs tables (support class, source component, source class) in the first context
    if ((rc = ensure(c0, c0->ws[W_RHS], (size_t)3 * Btot * sizeof(int)))) return rc;
    int *d_rhs_class = (int *)c0->ws[W_RHS].p, *d_src_comp = d_rhs_class + Btot, *d_src_class = d_src_comp + Btot;
    std::vector<int> h_rhs(3 * (size_t)Btot);
    std::vector<SolveSpec> specs(n);
    std::vector<SolveOut> outs(n);
    std::vector<int> maxit(n, 0), nb(n, 0);
    std::vector<long long> totit(n, 0);
    std::vector<double> worst(n, 0), truer(n, -1), solve_ms(n, 0);
    int nrel = 0;
    for (int r = 0; r < rounds; ++r) {
        int j0 = 0;
        for (int l = 0; l < n; ++l) {
            smpq_ctx *c = ctxs[l];
            for (int j = 0; j < Bl[l]; ++j) { // rhs r * Bl + j of lattice l: class (r Bl + j) / 12, component % 12
                const int g = r * Bl[l] + j;
                const int cl = g < N[l] ? g / 12 : -1;
                h_rhs[j0 + j] = cl;
                h_rhs[Btot + j0 + j] = g % 12;
                h_rhs[2 * Btot + j0 + j] = cl;
            }
            SolveSpec &sp = specs[l];
            sp = SolveSpec{};
            sp.B = Bl[l];
            sp.BC = BC;
            sp.prec = prec;
            sp.n_sup = nsup[l];
            sp.d_supsite = (const int *)c->ws[W_SUP].p;
            sp.d_rhs_class = d_rhs_class;
            sp.d_colour = (const int *)c->d_colour.p;
            sp.d_src_class = d_src_class;
            sp.d_src_comp = d_src_comp;
            sp.tpb_hi = shape.tpb_hi;
            sp.tpb_lo = shape.tpb_lo;
            sp.nr = 1;
            sp.staged = shape.staged;
            j0 += Bl[l];
        }
        cudaMemcpyAsync(d_rhs_class, h_rhs.data(), h_rhs.size() * sizeof(int), cudaMemcpyHostToDevice, st);
        if ((rc = multishift_solve_batch(ctxs, specs.data(), outs.data(), n))) {
            for (int l = 1; l < n; ++l) ctxs[l]->err = c0->err;
            return rc;
        }
        j0 = 0;
        for (int l = 0; l < n; ++l) {
            smpq_ctx *c = ctxs[l];
            const int *rc_l = d_rhs_class + j0, *comp_l = d_src_comp + j0;
            launch_add_c0b(nsup[l], Bl[l], BC, (const int *)c->ws[W_SUP].p, rc_l, comp_l, (const int *)c->d_colour.p,
                           c->c0, outs[l].y, st);
            launch_contract(c->geom, (const double *)c->U64.p, outs[l].y, nsup[l], Bl[l], BC, rc_l, comp_l,
                            (const int *)c->d_members.p, c->members, c->opt.kappa, (double2 *)c->ws[W_QTERM].p, st);
            c->launches += 2;
            maxit[l] = std::max(maxit[l], outs[l].iterations);
            totit[l] += outs[l].iterations;
            worst[l] = std::max(worst[l], outs[l].max_resid);
            if (outs[l].true_resid >= 0) truer[l] = std::max(truer[l], outs[l].true_resid);
            solve_ms[l] += outs[l].solve_ms;
            ++nb[l];
            j0 += Bl[l];
        }
        nrel += outs[0].reliable_updates;
    }
    // every lattice's q(x) and Q (all classes)
    for (int l = 0; l < n; ++l) {
        smpq_ctx *c = ctxs[l];
        if ((rc = ensure(c, c->ws[W_RHS], (size_t)c->n_classes * sizeof(int) + 4 * sizeof(double)))) return rc;
        int *d_classes = (int *)c->ws[W_RHS].p;
        double *d_tot = (double *)(((uintptr_t)(d_classes + c->n_classes) + 15) & ~(uintptr_t)15);
        std::vector<int> cls(c->n_classes);
        for (int k = 0; k < c->n_classes; ++k) cls[k] = k;
        cudaMemcpyAsync(d_classes, cls.data(), cls.size() * sizeof(int), cudaMemcpyHostToDevice, st);
        double *dq_re = q_re[l], *dq_im = q_im[l];
        if (!on_device) {
            if ((rc = ensure(c, c->ws[W_Q], 2 * (size_t)c->V * sizeof(double)))) return rc;
            dq_re = (double *)c->ws[W_Q].p;
            dq_im = dq_re + c->V;
        }
        launch_qsum((const double2 *)c->ws[W_QTERM].p, d_classes, c->n_classes, (const int *)c->d_members.p,
                    c->members, dq_re, dq_im, 0.5, st);
        launch_qtotal(dq_re, dq_im, nullptr, c->V, d_tot, st);
        c->launches += 2;
        double tot[2];
        cudaMemcpyAsync(tot, d_tot, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (!on_device) {
            cudaMemcpyAsync(q_re[l], dq_re, c->V * sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(q_im[l], dq_im, c->V * sizeof(double), cudaMemcpyDeviceToHost, st);
        }
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_check(c0, e, "uneven batch");
        c->last_Q = tot[0];
        if (Q) Q[l] = tot[0];
        if (stats) {
            smpq_stats &sx = stats[l];
            std::memset(&sx, 0, sizeof(sx));
            sx.n_rhs = N[l];
            sx.n_classes = c->n_classes;
            sx.n_batches = nb[l];
            sx.max_iterations = maxit[l];
            sx.total_iterations = totit[l];
            sx.reliable_updates = nrel;
            sx.max_resid = worst[l];
            sx.max_im_q = tot[1];
            sx.Q = tot[0];
            sx.q_round_dev = std::fabs(tot[0] - std::nearbyint(tot[0]));
            sx.solve_ms = solve_ms[l];
            sx.kernel_launches = c->launches; // (the shared solve's launches are on the first context)
            sx.rhs_tile = BC;
            sx.true_resid = truer[l];
            sx.tiles_per_block_hi = shape.tpb_hi;
            sx.tiles_per_block_lo = shape.tpb_lo;
            sx.cols_per_thread = 1;
            sx.shape_from_cache = from_cache;
            sx.staged = shape.staged;
        }
    }
    cudaEventRecord(c0->evB, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(c0, e, "uneven batch");
    float tms = 0;
    cudaEventElapsedTime(&tms, c0->evA, c0->evB);
    if (stats)
        for (int l = 0; l < n; ++l) stats[l].total_ms = tms;
    return cuda_check(c0, cudaGetLastError(), "uneven batch launch");
}

} // namespace

// ------------------------------------------------------------------ ABI
extern "C" {

int smpq_options_default(smpq_options *o) {
    if (!o) return SMPQ_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->kappa = 0.21;
    o->npoles = 14;
    o->tol = 1e-10;
    o->max_iter = 5000;
    o->precision = SMPQ_FP64;
    o->reliable_delta = 1e-3;
    for (int mu = 0; mu < 4; ++mu) o->bc[mu] = 1;
    o->rhs_block = 0;
    o->iters_per_check = 10;
    o->use_graphs = 1;
    o->profile = 0;
    o->switch_residual = 1e-3;
    o->autotune = 1;
    o->staging = -1;
    return SMPQ_OK;
}

int smpq_tune_cache_lookup(const char *path, const char *device, const int dims[4], int B, int precision,
                           int shape[5]) {
    if (!path || !device || !dims || !shape || B < 1) return SMPQ_EINVAL;
    FILE *f = std::fopen(path, "r");
    if (!f) return SMPQ_ESTATE;
    const std::string key = cache_key(device, dims, B, precision);
    char line[1024];
    int rc = SMPQ_ESTATE;
    while (std::fgets(line, sizeof line, f)) {
        if (std::strncmp(line, key.c_str(), key.size()) != 0) continue;
        int v[5];
        double ms;
        if (std::sscanf(line + key.size(), "%d %d %d %d %d|%lf", &v[0], &v[1], &v[2], &v[3], &v[4], &ms) == 6 &&
            (v[0] == 1 || v[0] == 12 || v[0] == 24 || v[0] == 48) && v[1] >= 1 && v[1] <= 64 && v[2] >= 1 &&
            v[2] <= 64 && (v[3] == 1 || v[3] == 2) && v[4] >= 0 && v[4] <= 3 && (!(v[4] & 1) || v[3] == 1)) {
            std::copy(v, v + 5, shape); // the last matching line wins
            rc = SMPQ_OK;
        }
    }
    std::fclose(f);
    return rc;
}

int smpq_tune_cache_store(const char *path, const char *device, const int dims[4], int B, int precision,
                          const int shape[5], double ms) {
    if (!path || !device || !dims || !shape || B < 1 || std::strchr(device, '|') || std::strchr(device, '\n'))
        return SMPQ_EINVAL;
    FILE *f = std::fopen(path, "a");
    if (!f) return SMPQ_EINVAL;
    const std::string key = cache_key(device, dims, B, precision);
    std::fprintf(f, "%s%d %d %d %d %d|%.6g\n", key.c_str(), shape[0], shape[1], shape[2], shape[3], shape[4], ms);
    std::fclose(f);
    return SMPQ_OK;
}

int smpq_create(smpq_ctx **out, int device, void *stream, const smpq_options *opt) {
    if (!out) return SMPQ_EINVAL;
    *out = nullptr;
    smpq_ctx *ctx = new (std::nothrow) smpq_ctx();
    if (!ctx) return SMPQ_ENOMEM;
    if (opt) ctx->opt = *opt;
    else smpq_options_default(&ctx->opt);
    ctx->tune_cache = ctx->opt.tune_cache ? ctx->opt.tune_cache : "";
    ctx->opt.tune_cache = nullptr; // the context keeps its own copy of the path
    int rc = validate_options(ctx, &ctx->opt);
    if (rc) { delete ctx; return rc; }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        delete ctx;
        return SMPQ_ECUDA;
    }
    ctx->device = device;
    DeviceGuard dg(device);
    ctx->user_stream = stream;
    e = cudaStreamCreate(&ctx->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev2);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->evA);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->evB);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return SMPQ_ECUDA;
    }
    ctx->ws.resize(W_COUNT);
    *out = ctx;
    return SMPQ_OK;
}

int smpq_destroy(smpq_ctx *ctx) {
    if (!ctx) return SMPQ_EINVAL;
    {
        DeviceGuard dg(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        for (auto &b : ctx->ws) release(b);
        release(ctx->U64);
        release(ctx->U32);
        release(ctx->Udf);
        release(ctx->d_err);
        release(ctx->Uh16);
        release(ctx->Ub16);
        release(ctx->d_colour);
        release(ctx->d_members);
        lowmodes_clear(ctx);
        cudaEventDestroy(ctx->ev0);
        cudaEventDestroy(ctx->ev1);
        cudaEventDestroy(ctx->ev2);
        cudaEventDestroy(ctx->evA);
        cudaEventDestroy(ctx->evB);
        for (cudaEvent_t ev : ctx->prof_ev) cudaEventDestroy(ev);
        cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
    return SMPQ_OK;
}

const char *smpq_last_error(const smpq_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int smpq_context_info(const smpq_ctx *ctx, int dims[4], int *device) {
    if (!ctx) return SMPQ_EINVAL;
    if (dims)
        for (int mu = 0; mu < 4; ++mu) dims[mu] = ctx->have_gauge ? ctx->dims[mu] : 0;
    if (device) *device = ctx->device;
    return SMPQ_OK;
}

int smpq_set_options(smpq_ctx *ctx, const smpq_options *opt) {
    if (!ctx || !opt) return SMPQ_EINVAL;
    int rc = validate_options(ctx, opt);
    if (rc) return rc;
    bool respec = opt->npoles != ctx->opt.npoles;
    ctx->opt = *opt;
    ctx->tune_cache = opt->tune_cache ? opt->tune_cache : "";
    ctx->opt.tune_cache = nullptr;
    if (ctx->have_gauge) set_geom(ctx);
    if (respec && ctx->have_spec) return smpq_set_spectrum(ctx, ctx->lmin2, ctx->lmax2);
    return SMPQ_OK;
}

int smpq_load_gauge(smpq_ctx *ctx, const int dims[4], const double *links, int on_device) {
    if (!ctx || !dims || !links) return SMPQ_EINVAL;
    long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2) return set_err(ctx, SMPQ_EINVAL, "every lattice extent must be >= 2");
        V *= dims[mu];
    }
    if (V > (1L << 28)) return set_err(ctx, SMPQ_EINVAL, "lattice volume above 2^28 sites");
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    cudaStreamSynchronize(ctx->stream);
    lowmodes_clear(ctx); // modes of the previous gauge field
    int rc;
    if ((rc = ensure(ctx, ctx->U64, (size_t)V * 36 * sizeof(double2)))) return rc;
    if ((rc = ensure(ctx, ctx->U32, (size_t)V * 36 * sizeof(float2)))) return rc;
    if ((rc = ensure(ctx, ctx->Udf, (size_t)V * 36 * sizeof(df64c)))) return rc;
    if ((rc = ensure(ctx, ctx->Uh16, (size_t)V * 24 * 4))) return rc;
    if ((rc = ensure(ctx, ctx->Ub16, (size_t)V * 24 * 4))) return rc;
    const double *src = links;
    if (on_device && (rc = check_device_ptr(ctx, links, "load_gauge links"))) return rc;
    if (!on_device) {
        if ((rc = ensure(ctx, ctx->ws[W_MISC], (size_t)V * 36 * sizeof(double2)))) return rc;
        cudaMemcpyAsync(ctx->ws[W_MISC].p, links, (size_t)V * 36 * sizeof(double2), cudaMemcpyHostToDevice,
                        ctx->stream);
        src = (const double *)ctx->ws[W_MISC].p;
    }
    for (int mu = 0; mu < 4; ++mu) ctx->dims[mu] = dims[mu];
    ctx->V = (int)V;
    set_geom(ctx);
    launch_pack_links(src, (double *)ctx->U64.p, (float *)ctx->U32.p, ctx->Udf.p, (int)V, ctx->stream);
    launch_pack_links12(src, ctx->Uh16.p, ctx->Ub16.p, (int)V, ctx->stream);
    if ((rc = ensure(ctx, ctx->ws[W_PART], 64))) return rc;
    double *derr = (double *)ctx->ws[W_PART].p;
    launch_su3_check((const double *)ctx->U64.p, (int)V, derr, ctx->stream);
    double err = 0;
    cudaMemcpyAsync(&err, derr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "load_gauge");
    if (!(err <= 1e-10)) {
        ctx->have_gauge = false;
        return set_err(ctx, SMPQ_ENOTSU3, "gauge field is not SU(3): max deviation " + std::to_string(err));
    }
    ctx->have_gauge = true;
    ctx->have_sources = false; // colouring depends on the lattice
    return SMPQ_OK;
}

int smpq_zolotarev(int npoles, double a, double b, double *c0, double *c, double *q, double *delta) {
    if (!c0 || !c || !q) return SMPQ_EINVAL;
    return zolotarev_coeffs(npoles, a, b, c0, c, q, delta);
}

int smpq_set_spectrum(smpq_ctx *ctx, double lmin2, double lmax2) {
    if (!ctx) return SMPQ_EINVAL;
    if (!(lmin2 > 0) || !(lmax2 > lmin2)) return set_err(ctx, SMPQ_EINVAL, "need 0 < lmin2 < lmax2");
    int n = ctx->opt.npoles;
    std::vector<double> c(n), q(n);
    double c0, d;
    int rc = zolotarev_coeffs(n, lmin2, lmax2, &c0, c.data(), q.data(), &d);
    if (rc) return set_err(ctx, rc, "zolotarev coefficients");
    ctx->lmin2 = lmin2;
    ctx->lmax2 = lmax2;
    ctx->c0 = c0;
    ctx->delta = d;
    ctx->zc = c;
    ctx->zq = q;
    ctx->have_spec = true;
    return SMPQ_OK;
}

int smpq_get_zolotarev(const smpq_ctx *ctx, double *c0, double *c, double *q, double *delta) {
    if (!ctx || !ctx->have_spec) return SMPQ_ESTATE;
    if (c0) *c0 = ctx->c0;
    if (c) std::copy(ctx->zc.begin(), ctx->zc.end(), c);
    if (q) std::copy(ctx->zq.begin(), ctx->zq.end(), q);
    if (delta) *delta = ctx->delta;
    return SMPQ_OK;
}

int smpq_measure_spectrum(smpq_ctx *ctx, int iters, double *lmin2, double *lmax2) {
    int rc = check_ctx(ctx, true, false, false);
    if (rc) return rc;
    if (iters < 4) return set_err(ctx, SMPQ_EINVAL, "need at least 4 Lanczos steps");
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    double lo, hi;
    if ((rc = lanczos_extremes(ctx, iters, &lo, &hi))) return rc;
    if (lmin2) *lmin2 = lo;
    if (lmax2) *lmax2 = hi;
    return smpq_set_spectrum(ctx, 0.98 * lo, 1.02 * hi);
}

int smpq_low_modes(smpq_ctx *ctx, int k, int block, double tol, int max_iter, double *evals, double *resid,
                   int *iterations) {
    int rc = check_ctx(ctx, true, true, false);
    if (rc) return rc;
    if (k < 1 || k > 43) return set_err(ctx, SMPQ_EINVAL, "low modes: need 1 <= k <= 43");
    int m = block;
    if (m <= 0) m = std::min(48, 12 * ((2 * k + 2 + 11) / 12));
    if (m < k + 5) m = 12 * ((k + 5 + 11) / 12);
    if (!(tol > 0)) tol = 1e-11;
    if (max_iter <= 0) max_iter = 200;
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    ctx->launches = 0;
    return lowmodes_compute(ctx, k, m, tol, max_iter, 20, evals, resid, iterations);
}

int smpq_get_low_modes(smpq_ctx *ctx, double *evecs, double *evals, int *k) {
    if (!ctx) return SMPQ_EINVAL;
    if (k) *k = ctx->lm_k;
    if (ctx->lm_k == 0) return SMPQ_OK;
    if (evals) std::copy(ctx->lm_val.begin(), ctx->lm_val.begin() + ctx->lm_k, evals);
    if (!evecs) return SMPQ_OK;
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    const int V = ctx->V, m = ctx->lm_m, kk = ctx->lm_k;
    const size_t n = (size_t)V * 12 * m;
    int rc = ensure(ctx, ctx->ws[W_OUT], n * sizeof(double2));
    if (rc) return rc;
    launch_from_tiled<double>(ctx->lm_vec.p, (double *)ctx->ws[W_OUT].p, V, m, 12, ctx->stream);
    std::vector<double> h(2 * n);
    cudaMemcpyAsync(h.data(), ctx->ws[W_OUT].p, n * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream);
    if ((rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "get_low_modes"))) return rc;
    for (size_t sc = 0; sc < (size_t)V * 12; ++sc)
        for (int j = 0; j < kk; ++j) {
            evecs[2 * (sc * kk + j)] = h[2 * (sc * m + j)];
            evecs[2 * (sc * kk + j) + 1] = h[2 * (sc * m + j) + 1];
        }
    return SMPQ_OK;
}

int smpq_clear_low_modes(smpq_ctx *ctx) {
    if (!ctx) return SMPQ_EINVAL;
    DeviceGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    lowmodes_clear(ctx);
    return SMPQ_OK;
}

int smpq_colour_sites(const int dims[4], int r, int mode, int *colour, int *n_classes) {
    if (!dims || !colour) return SMPQ_EINVAL;
    std::vector<int> col;
    int n = 0;
    int rc = colour_sites_host(dims, r, mode, col, &n, nullptr);
    if (rc) return rc;
    std::copy(col.begin(), col.end(), colour);
    if (n_classes) *n_classes = n;
    return SMPQ_OK;
}

int smpq_build_sources(smpq_ctx *ctx, int r, int mode, int *n_classes) {
    int rc = check_ctx(ctx, true, false, false);
    if (rc) return rc;
    std::string why;
    std::vector<int> col;
    int n = 0;
    if ((rc = colour_sites_host(ctx->dims, r, mode, col, &n, &why))) return set_err(ctx, rc, why);
    std::vector<int> count(n, 0);
    for (int c : col) ++count[c];
    int members = count[0];
    for (int c = 0; c < n; ++c)
        if (count[c] != members) return set_err(ctx, SMPQ_EINVAL, "colour classes of unequal size");
    std::vector<int> mem((size_t)n * members), fill(n, 0);
    for (int s = 0; s < ctx->V; ++s) mem[(size_t)col[s] * members + fill[col[s]]++] = s;
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    if ((rc = ensure(ctx, ctx->d_colour, (size_t)ctx->V * sizeof(int)))) return rc;
    if ((rc = ensure(ctx, ctx->d_members, mem.size() * sizeof(int)))) return rc;
    cudaMemcpyAsync(ctx->d_colour.p, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(ctx->d_members.p, mem.data(), mem.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "build_sources");
    ctx->colour.swap(col);
    ctx->r = r;
    ctx->mode = mode;
    ctx->n_classes = n;
    ctx->members = members;
    ctx->have_sources = true;
    if (n_classes) *n_classes = n;
    return SMPQ_OK;
}

static bool is_half(int precision) { return precision == SMPQ_FP16N || precision == SMPQ_BF16N; }

static const void *dslash_links(const smpq_ctx *ctx, int precision) {
    switch (precision) {
    case SMPQ_FP64: return ctx->U64.p;
    case SMPQ_FP32: return ctx->U32.p;
    case SMPQ_FP16N: return ctx->Uh16.p;
    default: return ctx->Ub16.p;
    }
}

// bytes of one field of B columns in the stand-alone D_W's format, rounded up
// to 256 so that a second field can follow it
static size_t dslash_field_bytes(const smpq_ctx *ctx, int precision, int B) {
    const size_t n = (size_t)ctx->V * 12 * B;
    const size_t b = is_half(precision) ? half_field_bytes(ctx->V, B) : n * (precision == SMPQ_FP64 ? 16 : 8);
    return (b + 255) / 256 * 256;
}

int smpq_dslash(smpq_ctx *ctx, const double *in, double *out, int B, int dagger, int precision, int on_device) {
    int rc = check_ctx(ctx, true, false, false);
    if (rc) return rc;
    if (!in || !out || B < 1) return set_err(ctx, SMPQ_EINVAL, "bad dslash arguments");
    if (precision != SMPQ_FP64 && precision != SMPQ_FP32 && !is_half(precision))
        return set_err(ctx, SMPQ_EINVAL, "bad precision");
    if (on_device && ((rc = check_device_ptr(ctx, in, "dslash in")) || (rc = check_device_ptr(ctx, out, "dslash out"))))
        return rc;
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    cudaStream_t st = ctx->stream;
    const size_t n = (size_t)ctx->V * 12 * B;
    const size_t fb = dslash_field_bytes(ctx, precision, B);
    if ((rc = ensure(ctx, ctx->ws[W_SRC], n * 16 + 2 * fb))) return rc;
    double *abi = (double *)ctx->ws[W_SRC].p;
    char *tin = (char *)ctx->ws[W_SRC].p + n * 16, *tout = tin + fb;
    const double *din = in;
    if (!on_device) {
        cudaMemcpyAsync(abi, in, n * 16, cudaMemcpyHostToDevice, st);
        din = abi;
    }
    const int BC = 1;
    const void *U = dslash_links(ctx, precision);
    double *dout = on_device ? out : abi;
    if (precision == SMPQ_FP64) {
        launch_to_tiled<double>(din, tin, ctx->V, B, BC, st);
        launch_dslash<double>(ctx->geom, U, tin, tout, B, BC, dagger, ctx->opt.kappa, st);
        launch_from_tiled<double>(tout, dout, ctx->V, B, BC, st);
    } else if (precision == SMPQ_FP32) {
        launch_to_tiled<float>(din, tin, ctx->V, B, BC, st);
        launch_dslash<float>(ctx->geom, U, tin, tout, B, BC, dagger, ctx->opt.kappa, st);
        launch_from_tiled<float>(tout, dout, ctx->V, B, BC, st);
    } else {
        launch_to_half(precision, din, tin, ctx->V, B, st);
        launch_dslash_half(precision, ctx->geom, U, tin, tout, B, dagger, ctx->opt.kappa, st);
        launch_from_half(precision, tout, dout, ctx->V, B, st);
    }
    if (!on_device) cudaMemcpyAsync(out, abi, n * 16, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "dslash");
    return cuda_check(ctx, cudaGetLastError(), "dslash launch");
}

int smpq_time_dslash(smpq_ctx *ctx, int B, int dagger, int precision, int reps, double *ms, double *bytes) {
    int rc = check_ctx(ctx, true, false, false);
    if (rc) return rc;
    if (B < 1 || reps < 1) return set_err(ctx, SMPQ_EINVAL, "bad time_dslash arguments");
    if (precision != SMPQ_FP64 && precision != SMPQ_FP32 && !is_half(precision))
        return set_err(ctx, SMPQ_EINVAL, "bad precision");
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    cudaStream_t st = ctx->stream;
    const size_t fb = dslash_field_bytes(ctx, precision, B);
    if ((rc = ensure(ctx, ctx->ws[W_SRC], 2 * fb))) return rc;
    char *tin = (char *)ctx->ws[W_SRC].p, *tout = tin + fb;
    cudaMemsetAsync(tin, 0x3F, 2 * fb, st);
    // the FP64 / FP32 tile: the widest of 48, 12 and 1 that divides B
    const int BC = B % 48 == 0 ? 48 : (B % 12 == 0 ? 12 : 1);
    const void *U = dslash_links(ctx, precision);
    // FP32 on tiles of 12 or more columns with staging 1: the neighbour sites staged in shared memory
    const bool staged = precision == SMPQ_FP32 && BC >= 12 && ctx->opt.staging == 1;
    if (staged) {
        if ((rc = ensure(ctx, ctx->d_err, 16))) return rc;
        cudaMemsetAsync(ctx->d_err.p, 0, 16, st);
    }
    cudaError_t le = cudaSuccess;
    auto launch = [&]() {
        if (precision == SMPQ_FP64) launch_dslash<double>(ctx->geom, U, tin, tout, B, BC, dagger, ctx->opt.kappa, st);
        else if (staged) {
            const cudaError_t e = launch_dslash_staged(ctx->geom, U, tin, tout, B, BC, dagger, ctx->opt.kappa,
                                                       (int *)ctx->d_err.p, st);
            if (e != cudaSuccess) le = e;
        } else if (precision == SMPQ_FP32) launch_dslash<float>(ctx->geom, U, tin, tout, B, BC, dagger, ctx->opt.kappa, st);
        else launch_dslash_half(precision, ctx->geom, U, tin, tout, B, dagger, ctx->opt.kappa, st);
    };
    launch();
    launch();
    cudaEventRecord(ctx->ev1, st);
    for (int k = 0; k < reps; ++k) launch();
    cudaEventRecord(ctx->ev2, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "time_dslash");
    if ((rc = cuda_check(ctx, le != cudaSuccess ? le : cudaGetLastError(), "time_dslash launch"))) return rc;
    if (staged) {
        int h = 0;
        if ((e = cudaMemcpy(&h, ctx->d_err.p, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_check(ctx, e, "time_dslash staging flag");
        if (h) return set_err(ctx, SMPQ_ECUDA, "a shared-memory staging wait of the FP32 D_W timed out");
    }
    float t = 0;
    if ((e = cudaEventElapsedTime(&t, ctx->ev1, ctx->ev2)) != cudaSuccess) return cuda_check(ctx, e, "time_dslash events");
    ctx->launches += reps + 2;
    const double V = ctx->V;
    const double spinor = precision == SMPQ_FP64 ? 192 : (precision == SMPQ_FP32 ? 96 : 52); // per site and rhs
    const double link = precision == SMPQ_FP64 ? 144 : (precision == SMPQ_FP32 ? 72 : 24);   // per stored link
    if (ms) *ms = (double)t / reps;
    if (bytes) *bytes = V * B * 2 * spinor + V * 4 * link;
    return SMPQ_OK;
}

int smpq_apply_dov(smpq_ctx *ctx, const double *in, double *out, int B, int on_device) {
    int rc = check_ctx(ctx, true, true, false);
    if (rc) return rc;
    if (!in || !out || B < 1) return set_err(ctx, SMPQ_EINVAL, "bad apply_dov arguments");
    if (on_device && ((rc = check_device_ptr(ctx, in, "apply_dov in")) || (rc = check_device_ptr(ctx, out, "apply_dov out"))))
        return rc;
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    cudaStream_t st = ctx->stream;
    const size_t n = (size_t)ctx->V * 12 * B;
    const bool project = ctx->lm_k > 0;
    if ((rc = ensure(ctx, ctx->ws[W_SRC], (project ? 4 : 3) * n * 16))) return rc;
    if ((rc = ensure(ctx, ctx->ws[W_RHS], 2 * (size_t)B * sizeof(int)))) return rc;
    double *abi = (double *)ctx->ws[W_SRC].p;
    double2 *b64 = (double2 *)(abi + 2 * n), *z = b64 + n, *bp = z + n;
    const double *din = in;
    if (!on_device) {
        cudaMemcpyAsync(abi, in, n * 16, cudaMemcpyHostToDevice, st);
        din = abi;
    }
    const int BC = 1;
    launch_to_tiled<double>(din, b64, ctx->V, B, BC, st);
    std::vector<double> wd; // V^dag b with the low modes treated exactly
    if (project && (rc = lowmodes_dov_project(ctx, b64, bp, B, wd, st))) return rc;
    const double2 *bsol = project ? bp : b64;
    cudaMemsetAsync(ctx->ws[W_RHS].p, 0, 2 * (size_t)B * sizeof(int), st); // every rhs in support class 0
    SolveSpec spec{};
    spec.B = B;
    spec.BC = BC;
    spec.prec = SMPQ_FP64;
    spec.full_support = 1;
    spec.n_sup = ctx->V;
    spec.d_supsite = nullptr;
    spec.d_rhs_class = (const int *)ctx->ws[W_RHS].p;
    spec.d_src_class = (const int *)ctx->ws[W_RHS].p;
    spec.d_src_comp = (const int *)ctx->ws[W_RHS].p + B;
    spec.d_colour = nullptr;
    spec.d_src_field = (const double *)bsol;
    SolveOut o;
    if ((rc = multishift_solve(ctx, spec, &o))) return rc;
    // y = c0 b + sum c_i x_i ; out = b + D_W y  (b -> b_perp in y, plus gamma_5 V sign V^dag b)
    launch_axpy(o.y, bsol, ctx->c0, n, st);
    launch_dslash<double>(ctx->geom, ctx->U64.p, o.y, z, B, BC, 0, ctx->opt.kappa, st);
    launch_axpy(z, b64, 1.0, n, st);
    if (project && (rc = lowmodes_dov_finish(ctx, z, B, wd, st))) return rc;
    double *dout = on_device ? out : abi;
    launch_from_tiled<double>(z, dout, ctx->V, B, BC, st);
    if (!on_device) cudaMemcpyAsync(out, abi, n * 16, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "apply_dov");
    return cuda_check(ctx, cudaGetLastError(), "apply_dov launch");
}

int smpq_compute_qx(smpq_ctx *ctx, double *q_re, double *q_im, int on_device, double *Q, smpq_stats *stats) {
    int rc = check_ctx(ctx, true, true, true);
    if (rc) return rc;
    if (!q_re || !q_im) return set_err(ctx, SMPQ_EINVAL, "null output");
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    std::vector<int> cls(ctx->n_classes);
    for (int c = 0; c < ctx->n_classes; ++c) cls[c] = c;
    rc = compute_classes(ctx, cls, q_re, q_im, on_device, stats, true);
    if (!rc && Q) *Q = ctx->last_Q;
    return rc;
}

int smpq_compute_qx_batch(smpq_ctx **ctxs, int n, double **q_re, double **q_im, int on_device, double *Q,
                          smpq_stats *stats) {
    if (!ctxs || n < 1 || !q_re || !q_im) return SMPQ_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !q_re[i] || !q_im[i]) return SMPQ_EINVAL;
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return set_err(ctxs[i], SMPQ_EINVAL, "a context appears twice in the batch");
    }
    // groups of at most 4 lattices share the launches of one solve
    for (int g0 = 0; g0 < n; g0 += 4) {
        const int m = std::min(4, n - g0);
        DeviceGuard dg(ctxs[g0]->device);
        for (int l = g0; l < g0 + m; ++l) StreamEntry se(ctxs[l], ctxs[l]->user_stream);
        // the other contexts' queued work precedes the group's solve on the first one's stream
        for (int l = g0 + 1; l < g0 + m; ++l) {
            cudaEventRecord(ctxs[l]->ev0, ctxs[l]->stream);
            cudaStreamWaitEvent(ctxs[g0]->stream, ctxs[l]->ev0, 0);
        }
        const int rc = compute_batch(ctxs + g0, m, q_re + g0, q_im + g0, on_device, Q ? Q + g0 : nullptr,
                                     stats ? stats + g0 : nullptr);
        if (rc) return rc;
    }
    return SMPQ_OK;
}

int smpq_trace_dwinv(smpq_ctx *ctx, double *t_re, double *t_im, int on_device, double *T, smpq_stats *stats) {
    int rc = check_ctx(ctx, true, false, true);
    if (rc) return rc;
    if (!t_re || !t_im) return set_err(ctx, SMPQ_EINVAL, "null output");
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    std::vector<int> cls(ctx->n_classes);
    for (int c = 0; c < ctx->n_classes; ++c) cls[c] = c;
    rc = compute_classes(ctx, cls, t_re, t_im, on_device, stats, true, 1);
    if (!rc && T) *T = ctx->last_Q;
    return rc;
}

int smpq_compute_qx_classes(smpq_ctx *ctx, const int *classes, int n, double *q_re, double *q_im, int on_device,
                            smpq_stats *stats) {
    int rc = check_ctx(ctx, true, true, true);
    if (rc) return rc;
    if (!classes || n < 1 || !q_re || !q_im) return set_err(ctx, SMPQ_EINVAL, "bad class list");
    std::vector<int> cls(classes, classes + n);
    std::vector<char> seen(ctx->n_classes, 0);
    for (int c : cls) {
        if (c < 0 || c >= ctx->n_classes || seen[c]) return set_err(ctx, SMPQ_EINVAL, "class id out of range or repeated");
        seen[c] = 1;
    }
    DeviceGuard dg(ctx->device);
    StreamEntry se(ctx, ctx->user_stream);
    return compute_classes(ctx, cls, q_re, q_im, on_device, stats, false);
}

} // extern "C"
