/*
 * smpq.h - C ABI of libsmpq: topological charge density q(x) = 1/2 tr(gamma_5 D_ov)(x,x)
 * estimated with symmetric multi-probing (SMP) sources on one GB300 GPU.
 *
 * Method (arXiv:1901.02211):
 *   D_ov = 1 + gamma_5 eps(gamma_5 D_W)                                (Sec. 2.1, Eq. 3)
 *   eps(H) = H (c0 + sum_{i=1}^{n} c_i / (H^2 + q_i)), H = gamma_5 D_W,
 *            H^2 = D_W^dag D_W, n = 14 Zolotarev poles                  (Sec. 2.1, Eq. 4)
 *   q(x) = 1/2 sum_{alpha,a} <psi(x,alpha,a)| gamma_5 D_ov |psi(x,alpha,a)>  (Eq. 5)
 *   the shifted systems (D_W^dag D_W + q_i) v_i = b are solved by CG     (Eqs. 6-8)
 *   SMP source phi_P(S, alpha, a) = sum_{y in S} psi(y, alpha, a)        (Sec. 2.2, Eq. 15)
 *   q^SMP(x) = sum_{alpha,a} psi(x,alpha,a) D~_ov phi_P(S(x,P),alpha,a),
 *              D~_ov = gamma_5 D_ov / 2                                  (Sec. 2.2, Eq. 16)
 *   colouring schemes P(m_x,m_y,m_z,m_t,mode), r_mu = n_mu/m_mu,
 *              mode 0 Normal, 1 Split, 2 Combine                          (Sec. 2.2, Eq. 19)
 *
 * Conventions:
 *   lattice dims = {nx, ny, nz, nt}, site index s = x + nx*(y + ny*(z + nz*t));
 *   D_W psi(x) = psi(x) - kappa sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                       + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)],
 *   chiral basis gamma_5 = diag(1, 1, -1, -1), bc[mu] = +1 periodic / -1 antiperiodic;
 *   complex numbers are interleaved (re, im) doubles;
 *   gauge field (host or device): double[V][4][3][3][2], U[s][mu][row][col];
 *   FP64 spinor fields at the ABI: double[V][4][3][B][2] (site, spin, colour, rhs).
 *
 * Errors: every call returns an smpq_status; nothing throws across the ABI.  On
 * error smpq_last_error(ctx) gives a message valid until the next call on ctx.
 * Device buffers: a buffer passed as device memory (on_device = 1, and both
 * buffers of smpq_dslash_noalloc) must be device or managed memory of the
 * context's GPU; anything else returns SMPQ_EINVAL before any launch.  Sizes
 * cannot be checked through a plain pointer: each call states what it reads
 * and writes, and a shorter buffer is the caller's error.
 * Ownership: caller buffers are only read or written during the call (device
 * buffers are used in stream order on the context's stream and the call
 * synchronises that stream before returning); the library never frees caller
 * memory and owns every device allocation it makes (released by smpq_destroy).
 * A context is not thread-safe; use one context per host thread.
 */
#ifndef SMPQ_H
#define SMPQ_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smpq_ctx smpq_ctx;

typedef enum {
    SMPQ_OK = 0,
    SMPQ_EINVAL = -1,     /* bad argument (sizes, scheme that does not tile, NULL) */
    SMPQ_ENOMEM = -2,     /* device allocation failed */
    SMPQ_ECUDA = -3,      /* CUDA runtime error (message in smpq_last_error) */
    SMPQ_ENOCONV = -4,    /* solver reached max_iter before every shift converged */
    SMPQ_EBREAKDOWN = -5, /* CG breakdown: <p, A p> <= 0 or non-finite */
    SMPQ_ETIMEOUT = -6,   /* reserved: a bounded device wait gave up */
    SMPQ_ENOTSU3 = -7,    /* gauge field is not SU(3) to 1e-10 */
    SMPQ_ESTATE = -8      /* call out of order (e.g. compute before load_gauge) */
} smpq_status;

typedef enum {
    SMPQ_FP64 = 0,  /* vectors, dslash and updates in FP64 (reference path) */
    SMPQ_FP32 = 1,  /* FP32 vectors and dslash with FP64 reliable updates, FP64 scalars */
    SMPQ_MIXED = 2, /* FP64-accurate iterations (float-float arithmetic on FP64-sized data)
                       until ||r|| <= switch_residual ||b||, then FP32 without residual
                       replacement; shifted directions in FP64 in the first phase and
                       FP32 in the second, y in FP64 throughout */
    SMPQ_FP16N = 3, /* spinor components stored in FP16 and scaled by one FP32 norm per site
                       and right-hand side, links stored as FP16 rows 0 and 1
                       (reconstruct-12), FP32 arithmetic.  smpq_dslash / smpq_time_dslash:
                       the stand-alone D_W in that format.  As a solver precision: the
                       SMPQ_FP32 iterations (FP64 reliable updates, FP32 residual and
                       shifted directions) with D_W's input p and output t in that
                       format; the shifted systems then keep an error floor near the
                       format's rounding (about 1e-4 relative), far above FP32's. */
    SMPQ_BF16N = 4  /* as SMPQ_FP16N with BF16 storage (floor near 1e-3 relative) */
} smpq_precision;

typedef struct {
    double kappa;          /* Wilson hopping parameter (Sec. 2.1: 0.21) */
    int npoles;            /* Zolotarev poles (Sec. 2.1: 14); 1..32 */
    double tol;            /* per-shift relative residual |zeta_i| ||r|| / ||b|| */
    int max_iter;          /* CG iteration cap */
    int precision;         /* smpq_precision */
    double reliable_delta; /* FP32 path: replace the residual when ||r|| < delta * max ||r||
                              (SMPQ_FP16N / SMPQ_BF16N use at least 0.1) */
    int bc[4];             /* fermion boundary factors per direction */
    int rhs_block;         /* right-hand sides per solve batch (multiple of 12; 0 = automatic) */
    int iters_per_check;   /* CG iterations launched between host convergence checks */
    int use_graphs;        /* capture those iterations in a CUDA graph */
    int profile;           /* time every D_W / D_W^dag launch of the solver with CUDA events */
    double switch_residual; /* SMPQ_MIXED: relative residual at which FP64 iterations hand over to FP32 */
    int autotune;           /* time the D_W launch shapes (RHS tile 12, 24, 48; tiles per block 1, 2,
                               4, 8; FP32 columns per thread 1, 2; neighbours staged in shared
                               memory or not, per phase) on the first solve of each batch shape,
                               and use the fastest */
    int full_support;       /* q(x): keep the shifted directions on every site instead of only where
                               z = D_W y is read (the ablation of that restriction; same result,
                               14 full-lattice vectors per source) */
    int true_residual;      /* SMPQ_FP64 / SMPQ_MIXED, the base system's true residual
                               |b - (H^2 + s0) x| / |b| (smpq_stats.true_resid):
                               0: not computed (no base solution is kept);
                               1: x is accumulated (two more whole-lattice fields per source)
                                  and the residual recomputed with FP64 accuracy at the end;
                               2 (SMPQ_MIXED): as 1, and the base system is then iterated on from
                                  its true residual until that is below tol (the FP32 phase's
                                  rounding leaves it at a few times 1e-8 otherwise, at the
                                  default switch_residual).  The FP32 and half
                                  paths always report it from their last reliable update. */
    const char *tune_cache; /* path of a text file of tuned launch shapes (NULL: none): read before
                               tuning a new shape, appended after (see smpq_tune_cache_lookup).  The
                               context copies the path. */
    int staging;            /* D_W launches of the FP32 iterations (SMPQ_FP32, the second phase of
                               SMPQ_MIXED) and of the float-float ones (the first phase of
                               SMPQ_MIXED) with the neighbour sites staged in shared memory by bulk
                               asynchronous copies, one column per thread: -1 the autotuner chooses
                               per phase (plain loads when autotune is 0), 0 never, 1 always (RHS
                               tiles of 12 columns or more).  The stand-alone FP32 D_W of
                               smpq_time_dslash stages only when this is 1. */
} smpq_options;

typedef struct {
    int n_rhs;              /* right-hand sides solved by the last call */
    int n_classes;          /* colour classes processed */
    int n_batches;          /* solve batches */
    int max_iterations;     /* largest CG iteration count of any right-hand side */
    long long total_iterations; /* sum over batches of the batch iteration count */
    int reliable_updates;   /* FP64 residual replacements (FP32 path) */
    double max_resid;       /* largest final recursive residual |zeta_i| ||r|| / ||b|| */
    double max_im_q;        /* max |Im q^SMP(x)| over processed sites */
    double Q;               /* sum_x Re q(x) over the processed sites */
    double solve_ms;        /* device time of the solves (CUDA events) */
    double total_ms;        /* device time of the whole call */
    long long kernel_launches; /* CUDA kernels launched by the call (graph nodes included) */
    double dslash_ms;       /* profile: summed time of the t = D_W p launches */
    long long dslash_launches;
    double update_ms;       /* profile: summed time of the r -= alpha (D_W^dag t + s0 p) launches */
    long long update_launches;
    /* profile, FP64-accurate iterations (SMPQ_FP64, and the first phase of
       SMPQ_MIXED); the four fields above then count FP32 iterations only */
    double dslash_hi_ms;
    long long dslash_hi_launches;
    double update_hi_ms;
    long long update_hi_launches;
    int rhs_tile;           /* RHS tile width the solves used (autotuned or fixed) */
    double q_round_dev;     /* |Q - round(Q)| of the processed sites (the charge is an integer) */
    double true_resid;      /* largest true relative residual |b - (H^2 + s0) x| / |b| of the base
                               (smallest) shift, recomputed with FP64 accuracy after the solve; -1
                               when not computed (SMPQ_FP64 / SMPQ_MIXED with true_residual 0) */
    int tiles_per_block_hi; /* launch shape of the D_W kernels (autotuned): tiles per block of the */
    int tiles_per_block_lo; /*   FP64-accurate and of the FP32 / half-storage iterations, */
    int cols_per_thread;    /*   FP32 columns per thread (1 or 2), */
    int shape_from_cache;   /*   1 if the shape came from the tune_cache file, */
    int staged;             /*   D_W launches that staged the neighbour sites in shared memory
                                 (bulk asynchronous copies; one column per thread): bit 0 the FP32
                                 iterations, bit 1 the float-float ones */
} smpq_stats;

/* Fill *opt with the paper's parameters: kappa 0.21, 14 poles, tol 1e-10,
 * max_iter 5000, FP64, reliable_delta 1e-3, periodic bc, automatic batching,
 * 10 iterations per check, graphs on, profiling off, switch_residual 1e-3,
 * autotuning on, no true-residual accumulation, no tuning cache file, staging
 * chosen by the autotuner (-1). */
int smpq_options_default(smpq_options *opt);

/* Create a context on CUDA device `device` using `stream` (a cudaStream_t, e.g.
 * torch.cuda.current_stream().cuda_stream; NULL = the legacy default stream).
 * *out receives the context; options are copied. */
int smpq_create(smpq_ctx **out, int device, void *stream, const smpq_options *opt);
int smpq_destroy(smpq_ctx *ctx);
const char *smpq_last_error(const smpq_ctx *ctx);

/* The context's lattice and GPU: dims (nullable) receives {nx, ny, nz, nt} of
 * the loaded gauge field (zeros before smpq_load_gauge), *device (nullable)
 * the CUDA device index.  Not in the paper: callers use it to size and place
 * the buffers of the calls below. */
int smpq_context_info(const smpq_ctx *ctx, int dims[4], int *device);

/* Change the options of an existing context (kappa/bc changes take effect on
 * the next call; the gauge field and spectrum stay loaded). */
int smpq_set_options(smpq_ctx *ctx, const smpq_options *opt);

/* Load the gauge field U_mu(x) (Sec. 2.1: the links of D_W).  dims: {nx,ny,nz,nt},
 * each >= 2 and V <= 2^28; links: double[V][4][3][3][2], host (on_device=0) or
 * device memory; copied and packed into the context's FP64 and FP32 link arrays.
 * SMPQ_ENOTSU3 if any link deviates from unitarity or det = 1 by more than 1e-10. */
int smpq_load_gauge(smpq_ctx *ctx, const int dims[4], const double *links, int on_device);

/* Set the Zolotarev interval [a, b] = [lmin2, lmax2] of H_W^2 and compute the
 * coefficients (Eq. 4).  0 < lmin2 < lmax2. */
int smpq_set_spectrum(smpq_ctx *ctx, double lmin2, double lmax2);

/* Estimate the extreme eigenvalues of H_W^2 by `iters` Lanczos steps (CG
 * coefficients on a seeded random vector) and set the interval to
 * [0.98 lmin2, 1.02 lmax2] (the paper does not say how the interval is chosen).
 * Outputs (nullable) receive the unwidened Ritz values. */
int smpq_measure_spectrum(smpq_ctx *ctx, int iters, double *lmin2, double *lmax2);

/* Low modes of H_W = gamma_5 D_W treated exactly in the sign function (a
 * standard overlap technique; the paper evaluates eps(H_W) of Eq. 4 with the
 * rational alone and mentions low modes only of D_ov, end of Sec. 3):
 *   eps(H) = sum_{j<k} sign(lambda_j) v_j v_j^dag + H R(H^2) (1 - sum_j v_j v_j^dag).
 * Computes the k + 1 eigenpairs of H_W of smallest |lambda| by Chebyshev-
 * filtered subspace iteration on H_W^2 (block of `block` vectors, a multiple of
 * 12 up to 48; 0 chooses about 2k + 2), FP64, until ||H v - lambda v|| <= tol
 * (<= 0: 1e-11) for all k + 1, at most max_iter filter steps (<= 0: 200).
 * Needs a gauge field and a spectral interval whose upper end bounds H_W^2.
 * evals, resid (nullable): k + 1 doubles, signed lambda_j ordered by |lambda|
 * and residual norms; *iterations (nullable): filter steps.  From then on,
 * smpq_compute_qx[_classes] and smpq_apply_dov treat the first k modes exactly:
 * the solves run on the projected sources and q^SMP(x) gains the low-mode term
 * 1/2 sum_{alpha,a} sum_j sign(lambda_j) v_j(x,alpha,a) (v_j^dag b_{alpha,a}).
 * The rational still follows the context's interval: set it next with
 * smpq_set_spectrum(ctx, 0.98 * evals[k]^2, b) to shorten it.  Loading a gauge
 * field or smpq_clear_low_modes drops the modes.  1 <= k <= 43; SMPQ_ENOCONV if
 * not converged (no modes kept). */
int smpq_low_modes(smpq_ctx *ctx, int k, int block, double tol, int max_iter, double *evals, double *resid,
                   int *iterations);

/* The modes in use: *k (nullable) = their number (0: none); evals (nullable):
 * k doubles; evecs (nullable): host double[V][4][3][k][2], orthonormal. */
int smpq_get_low_modes(smpq_ctx *ctx, double *evecs, double *evals, int *k);

/* Drop the low modes: back to the rational on the whole spectrum. */
int smpq_clear_low_modes(smpq_ctx *ctx);

/* Zolotarev coefficients of R(x) = c0 + sum_i c[i]/(x + q[i]) ~ 1/sqrt(x) on
 * [a, b] (Eq. 4), type (npoles, npoles), q ascending; *delta = max relative
 * error.  Pure host computation; c and q hold npoles doubles. */
int smpq_zolotarev(int npoles, double a, double b, double *c0, double *c, double *q, double *delta);

/* Coefficients currently used by the context (after set/measure_spectrum). */
int smpq_get_zolotarev(const smpq_ctx *ctx, double *c0, double *c, double *q, double *delta);

/* Choose the colouring scheme (Sec. 2.2): same-colour sites every r sites in
 * each direction (r_mu = r), mode 0 Normal / 1 Split / 2 Combine.  SMPQ_EINVAL
 * if r does not divide every n_mu, if mode 1 and some n_mu/r is odd, or if
 * mode 2 and r is odd.  *n_classes (nullable) = N_p; the solve count is 12 N_p. */
int smpq_build_sources(smpq_ctx *ctx, int r, int mode, int *n_classes);

/* Host-side colouring only (no GPU work): colour of every site, int[V].  Same
 * validation as smpq_build_sources. */
int smpq_colour_sites(const int dims[4], int r, int mode, int *colour, int *n_classes);

/* D_W (or gamma_5 D_W gamma_5 = D_W^dag if dagger) applied to B fields
 * (Sec. 2.1, Eq. 3), computed in `precision`: SMPQ_FP64 or SMPQ_FP32 kernels,
 * or SMPQ_FP16N / SMPQ_BF16N (the input is rounded to the half format on the
 * device, the result leaves the kernel in that format and is widened back to
 * FP64).  in/out FP64 at the ABI: double[V][4][3][B][2], host or device
 * (on_device).  SMPQ_EINVAL for SMPQ_MIXED or an unknown precision. */
int smpq_dslash(smpq_ctx *ctx, const double *in, double *out, int B, int dagger, int precision, int on_device);

/* Average device time of one stand-alone D_W launch (the kernel behind
 * smpq_dslash, Sec. 2.1, Eq. 3) on B right-hand sides held in `precision`
 * (SMPQ_FP64, SMPQ_FP32, SMPQ_FP16N or SMPQ_BF16N), in the RHS tile the
 * library picks for B.  The input and output fields are scratch in the
 * context's workspace, set once to the byte 0x3F (finite values in every
 * format; the values do not change the work).  Two untimed launches, then
 * `reps` (>= 1) launches back to back on the context's stream between two
 * CUDA events.  *ms (nullable): average milliseconds per launch; *bytes
 * (nullable): algorithmic bytes of one launch, V * B * (spinor bytes read +
 * written per site and rhs) + V * 4 * (bytes per stored link).  Needs a gauge
 * field (SMPQ_ESTATE otherwise). */
int smpq_time_dslash(smpq_ctx *ctx, int B, int dagger, int precision, int reps, double *ms, double *bytes);

/* Allocation-free variant of smpq_dslash (the paper has no counterpart; this
 * is a service for callers of this library).  Some callers cannot call
 * cudaMalloc: code whose device memory is owned by another allocator that must
 * see every allocation (a framework's caching allocator), or latency-critical
 * loops where cudaMalloc/cudaFree would synchronise the device.  This call
 * allocates nothing: in and out are caller-owned DEVICE buffers in the layout
 * of smpq_dslash, and the kernel's scratch (tiled copies of in and out) lives
 * in a file-scope device array of 32 MiB that every GPU which loads the
 * library holds until the process exits.
 *   - Limit: 2 * V * 12 * B * e bytes <= 32 MiB, e = 16 (FP64) or 8 (FP32);
 *     larger requests return SMPQ_EINVAL with the sizes in smpq_last_error.
 *   - The first call on a device looks up the device address of the scratch
 *     array (cudaGetSymbolAddress, with that device current); make that first
 *     call before any stream capture on the device.
 *   - Every call on a device shares the same scratch.  Each call overwrites all
 *     of the scratch it uses (nothing has to start at zero) and synchronises
 *     the context's stream before returning, but calls from different
 *     contexts or host threads that overlap on the GPU race on the scratch.
 * Requires a loaded gauge field (SMPQ_ESTATE otherwise). */
int smpq_dslash_noalloc(smpq_ctx *ctx, const double *in, double *out, int B, int dagger, int precision);

/* out = D_ov in = in + D_W R(H^2) in (Eqs. 3-4 with gamma_5^2 = 1), B fields,
 * FP64 multi-shift CG over the full lattice.  Layout as smpq_dslash. */
int smpq_apply_dov(smpq_ctx *ctx, const double *in, double *out, int B, int on_device);

/* q^SMP(x) for every site with the scheme of smpq_build_sources (Eq. 16):
 * q_re, q_im: double[V] (host or device), Q (nullable): sum_x Re q(x).
 * With r = n_mu in every direction every set is one site and the result is
 * the exact point-source q(x) of Eq. 5. */
int smpq_compute_qx(smpq_ctx *ctx, double *q_re, double *q_im, int on_device, double *Q, smpq_stats *stats);

/* As smpq_compute_qx for the listed colour classes only (sampled checks,
 * checkpoint/resume).  Sites of other classes are left untouched in q_re/q_im. */
int smpq_compute_qx_classes(smpq_ctx *ctx, const int *classes, int n, double *q_re, double *q_im, int on_device,
                            smpq_stats *stats);

/* Uneven batch: q^SMP(x) for n lattices of different sizes and schemes, one
 * context each (distinct contexts on one device, each with its gauge field,
 * spectrum and colouring loaded; one precision and pole count for all; no
 * low-mode projection, full_support or rhs_block = 1).  Up to four lattices
 * share one solve: every CG iteration is the same three kernel launches for
 * all of them (each RHS tile carries its lattice's geometry, links and
 * rational), issued on the first context's stream, whose workspace holds the
 * fields.  Their sources run in rounds sized to the device memory, each round
 * taking about the same share of every lattice's sources.  Larger n runs in
 * groups of four.  The default launch shape is used (no autotuning).
 * q_re[i], q_im[i]: double[V_i]; Q and stats (nullable): arrays of n.
 * Returns the first non-OK status (its message is on the first context). */
int smpq_compute_qx_batch(smpq_ctx **ctxs, int n, double **q_re, double **q_im, int on_device, double *Q,
                          smpq_stats *stats);

/* SMP estimate of the diagonal of D_W^{-1} and of Tr D_W^{-1} (the paper's
 * closing remark, Sec. 4: the same sources applied to the ultra-local Wilson
 * operator): t(x) = sum_{alpha,a} <psi(x,alpha,a)| D_W^{-1} |phi_P(S(x),alpha,a)>,
 * *T = sum_x Re t(x).  D_W^{-1} b = (D_W^dag D_W)^{-1} D_W^dag b by CG in the
 * context's precision.  Needs a gauge field and a colouring scheme (no
 * spectrum).  t_re, t_im: double[V], host or device. */
int smpq_trace_dwinv(smpq_ctx *ctx, double *t_re, double *t_im, int on_device, double *T, smpq_stats *stats);

/* The autotuner's cache file (host only; not part of the paper's method).
 * A shape is {RHS tile width (1, 12, 24, 48), tiles per block of the
 * FP64-accurate D_W launches, tiles per block of the FP32 / half-storage ones,
 * FP32 columns per thread (1, 2), neighbours staged in shared memory (bit 0
 * the FP32 iterations, only with one column; bit 1 the float-float ones)},
 * keyed by a device string (as the library writes it: "<name>/<SMs>sm"), the
 * lattice dims, the batch B and the precision.  One line per entry:
 *   smpq-tune-2|<device>|<nx> <ny> <nz> <nt>|<B>|<precision>|<bc> <tpb_hi> <tpb_lo> <nr> <staged>|<ms>
 * lookup: SMPQ_OK and shape[5] filled from the last matching well-formed line,
 * SMPQ_ESTATE if the file is missing or has no such line, SMPQ_EINVAL for
 * NULL arguments.  store: appends one line (ms = the tuner's estimate per
 * iteration pair); SMPQ_EINVAL if the file cannot be opened or the device
 * string holds '|' or a newline.  Neither call takes a lock: processes that
 * tune the same shape at once both append, and the last line wins. */
int smpq_tune_cache_lookup(const char *path, const char *device, const int dims[4], int B, int precision,
                           int shape[5]);
int smpq_tune_cache_store(const char *path, const char *device, const int dims[4], int B, int precision,
                          const int shape[5], double ms);

/* Measured arithmetic peak of GPU `device` (not part of the paper's method: the
 * denominator of the ALU rooflines the solver's FP64-accurate kernels are
 * reported against).  kind 0: FP32 fused multiply-adds as scalar instructions,
 * 1: FP32 in packed two-lane instructions (sm_100 and later), 2: FP64 fused
 * multiply-adds.  *ops_per_s = lane operations (one multiply-add each) per
 * second, best of three launches of 8 independent chains per thread on 8
 * blocks of 256 threads per SM.  Runs on a stream of its own; allocates and
 * frees one small device buffer.  SMPQ_EINVAL for an unknown kind,
 * SMPQ_ECUDA for a bad device or a CUDA error. */
int smpq_alu_peak(int device, int kind, double *ops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* SMPQ_H */
