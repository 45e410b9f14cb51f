// Link packing, SU(3) check, layout conversion and the stand-alone Wilson
// dslash D_W / D_W^dag (Sec. 2.1, around Eq. 3) used by smpq_dslash.
#include <string>

#include "smpq_internal.cuh"
#include "stage.cuh"
#include "wilson.cuh"

// ------------------------------------------------------------------ links
// U_aos: double[V][4][3][3][2] -> U64/U32: [(mu * V + s) * 9 + e] complex
__global__ void pack_links_kernel(const double2 *__restrict__ Uaos, double2 *__restrict__ U64,
                                  float2 *__restrict__ U32, df64c *__restrict__ Udf, int V) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)V * 36) return;
    int s = (int)(i / 36), k = (int)(i % 36); // k = mu*9 + e
    double2 u = Uaos[i];
    size_t o = ((size_t)(k / 9) * V + s) * 9 + (k % 9);
    U64[o] = u;
    U32[o] = make_float2((float)u.x, (float)u.y);
    Udf[o] = df64c{df64(u.x), df64(u.y)};
}

void launch_pack_links(const double *U_aos, double *U64, float *U32, void *Udf, int V, cudaStream_t st) {
    long n = (long)V * 36;
    pack_links_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double2 *)U_aos, (double2 *)U64,
                                                                     (float2 *)U32, (df64c *)Udf, V);
}

// max over links of max(|U U^dag - 1|, |det U - 1|), as the bit pattern of a
// non-negative double (ordered like unsigned integers) for atomicMax.
__global__ void su3_check_kernel(const double2 *__restrict__ U, int V, unsigned long long *out) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    double err = 0;
    if (i < (long)V * 4) {
        int s = (int)(i / 4), mu = (int)(i % 4);
        double2 u[9];
        for (int e = 0; e < 9; ++e) u[e] = U[((size_t)mu * V + s) * 9 + e];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double2 t = make_double2(0, 0);
                for (int k = 0; k < 3; ++k) t = cfmac(u[b * 3 + k], u[a * 3 + k], t); // (U U^dag)_ab
                double d = sqrt((t.x - (a == b)) * (t.x - (a == b)) + t.y * t.y);
                err = fmax(err, d);
            }
        // det by cofactor expansion along row 0
        double2 m0 = csub(cmul(u[4], u[8]), cmul(u[5], u[7]));
        double2 m1 = csub(cmul(u[3], u[8]), cmul(u[5], u[6]));
        double2 m2 = csub(cmul(u[3], u[7]), cmul(u[4], u[6]));
        double2 det = cadd(csub(cmul(u[0], m0), cmul(u[1], m1)), cmul(u[2], m2));
        err = fmax(err, sqrt((det.x - 1) * (det.x - 1) + det.y * det.y));
        if (!(err == err)) err = 1e300; // NaN
    }
    // block max then one atomic
    __shared__ double sm[256];
    sm[threadIdx.x] = err;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + st]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sm[0]));
}

void launch_su3_check(const double *U64, int V, double *dev_maxerr, cudaStream_t st) {
    cudaMemsetAsync(dev_maxerr, 0, sizeof(double), st);
    long n = (long)V * 4;
    su3_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double2 *)U64, V,
                                                                   (unsigned long long *)dev_maxerr);
}

// ------------------------------------------------------------------ layout conversion
// ABI [V][12][B] double2  <->  tiled [j/BC][V][12][BC] of complex T
template <typename T>
__global__ void to_tiled_kernel(const double2 *__restrict__ in, typename cplx_t<T>::type *__restrict__ out, int V,
                                int B, int BC) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)V * 12 * B) return;
    int j = (int)(i % B);
    long r = i / B;
    int c = (int)(r % 12);
    int s = (int)(r / 12);
    double2 v = in[i];
    size_t o = (((size_t)(j / BC) * V + s) * 12 + c) * BC + (j % BC);
    out[o] = mkc<typename cplx_t<T>::type>(v.x, v.y);
}

template <typename T>
__global__ void from_tiled_kernel(const typename cplx_t<T>::type *__restrict__ in, double2 *__restrict__ out, int V,
                                  int B, int BC) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)V * 12 * B) return;
    int j = (int)(i % B);
    long r = i / B;
    int c = (int)(r % 12);
    int s = (int)(r / 12);
    size_t o = (((size_t)(j / BC) * V + s) * 12 + c) * BC + (j % BC);
    typename cplx_t<T>::type v = in[o];
    out[i] = make_double2((double)v.x, (double)v.y);
}

template <typename T> void launch_to_tiled(const double *in, void *out, int V, int B, int BC, cudaStream_t st) {
    long n = (long)V * 12 * B;
    to_tiled_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double2 *)in,
                                                                     (typename cplx_t<T>::type *)out, V, B, BC);
}
template <typename T> void launch_from_tiled(const void *in, double *out, int V, int B, int BC, cudaStream_t st) {
    long n = (long)V * 12 * B;
    from_tiled_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const typename cplx_t<T>::type *)in,
                                                                       (double2 *)out, V, B, BC);
}
template void launch_to_tiled<double>(const double *, void *, int, int, int, cudaStream_t);
template void launch_to_tiled<float>(const double *, void *, int, int, int, cudaStream_t);
template void launch_from_tiled<double>(const void *, double *, int, int, int, cudaStream_t);
template void launch_from_tiled<float>(const void *, double *, int, int, int, cudaStream_t);

// ------------------------------------------------------------------ stand-alone dslash
template <typename T, bool DAG, int BC>
__global__ void __launch_bounds__(TileMap<BC>::THREADS)
    dslash_kernel(Geom g, const typename cplx_t<T>::type *__restrict__ U, const typename cplx_t<T>::type *__restrict__ in,
                  typename cplx_t<T>::type *__restrict__ out, T kappa) {
    typedef typename cplx_t<T>::type C;
    int s = blockIdx.x * TileMap<BC>::SPB + threadIdx.x / BC;
    int jj = threadIdx.x % BC;
    if (s >= g.V) return;
    size_t base = (size_t)blockIdx.y * 12 * g.V * BC + jj;
    const C *pin = in + base;
    C acc[12][1];
    wilson_hop<T, DAG, BC>(g, U, pin, s, acc);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        size_t o = ((size_t)s * 12 + c) * BC;
        C v = pin[o];
        v.x -= kappa * acc[c][0].x;
        v.y -= kappa * acc[c][0].y;
        out[base + o] = v;
    }
}

template <typename T, int BC>
static void dslash_bc(const Geom &g, const void *U, const void *in, void *out, int B, int dagger, double kappa,
                      cudaStream_t st) {
    typedef typename cplx_t<T>::type C;
    dim3 grid((g.V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB, B / BC);
    if (dagger)
        dslash_kernel<T, true, BC><<<grid, TileMap<BC>::THREADS, 0, st>>>(g, (const C *)U, (const C *)in, (C *)out,
                                                                           (T)kappa);
    else
        dslash_kernel<T, false, BC><<<grid, TileMap<BC>::THREADS, 0, st>>>(g, (const C *)U, (const C *)in, (C *)out,
                                                                            (T)kappa);
}

// The FP32 D_W with the neighbour sites staged in shared memory (stage.cuh):
// out = in - kappa hop(in), tpb lattice tiles per block.
template <bool DAG, int BC>
__global__ void __launch_bounds__(TileMap<BC>::THREADS, 3)
    dslash_staged_kernel(Geom g, const float2 *__restrict__ U, const float2 *__restrict__ in, float2 *__restrict__ out,
                         double kd, int tpb, int *err) {
    typedef TileMap<BC> TM;
    extern __shared__ __align__(128) unsigned char dsm[];
    const int jj = threadIdx.x % BC;
    const size_t tb = (size_t)blockIdx.y * 12 * g.V * BC;
    const int ntiles = (g.V + TM::SPB - 1) / TM::SPB;
    const int tile0 = blockIdx.x * tpb, ntb = min(ntiles, tile0 + tpb) - tile0;
    const float kappa = (float)kd;
    stage::Runner<DAG, BC, stage::NSTAGE> run(dsm, g, U, in + tb, tile0, ntb, err);
    for (int tl = 0; tl < ntb; ++tl) {
        const int s = (tile0 + tl) * TM::SPB + threadIdx.x / BC;
        const bool valid = s < g.V;
        float2 acc[12][1];
        run.hops(tl, s, valid, acc);
        if (!valid) continue;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t o = tb + ((size_t)s * 12 + c) * BC + jj;
            float2 v = in[o];
            v.x -= kappa * acc[c][0].x;
            v.y -= kappa * acc[c][0].y;
            out[o] = v;
        }
    }
}

template <int BC>
static cudaError_t dslash_staged_bc(const Geom &g, const void *U, const void *in, void *out, int B, int dagger,
                                    double kappa, int *err, cudaStream_t st) {
    constexpr int TPB_ST = 4; // lattice tiles per block
    const int bytes = (int)stage::Dims<BC, stage::NSTAGE>::SMEM;
    static bool attrs = false;
    if (!attrs) {
        cudaError_t e = cudaFuncSetAttribute(dslash_staged_kernel<false, BC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(dslash_staged_kernel<true, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     bytes);
        if (e != cudaSuccess) return e;
        attrs = true;
    }
    const int ntiles = (g.V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    const dim3 grid((ntiles + TPB_ST - 1) / TPB_ST, B / BC);
    if (dagger)
        dslash_staged_kernel<true, BC><<<grid, TileMap<BC>::THREADS, bytes, st>>>(
            g, (const float2 *)U, (const float2 *)in, (float2 *)out, kappa, TPB_ST, err);
    else
        dslash_staged_kernel<false, BC><<<grid, TileMap<BC>::THREADS, bytes, st>>>(
            g, (const float2 *)U, (const float2 *)in, (float2 *)out, kappa, TPB_ST, err);
    return cudaSuccess;
}

cudaError_t launch_dslash_staged(const Geom &g, const void *U, const void *in, void *out, int B, int BC, int dagger,
                                 double kappa, int *err, cudaStream_t st) {
    switch (BC) {
    case 12: return dslash_staged_bc<12>(g, U, in, out, B, dagger, kappa, err, st);
    case 24: return dslash_staged_bc<24>(g, U, in, out, B, dagger, kappa, err, st);
    case 48: return dslash_staged_bc<48>(g, U, in, out, B, dagger, kappa, err, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
void launch_dslash(const Geom &g, const void *U, const void *in, void *out, int B, int BC, int dagger, double kappa,
                   cudaStream_t st) {
    switch (BC) {
    case 1: dslash_bc<T, 1>(g, U, in, out, B, dagger, kappa, st); break;
    case 4: dslash_bc<T, 4>(g, U, in, out, B, dagger, kappa, st); break;
    case 12: dslash_bc<T, 12>(g, U, in, out, B, dagger, kappa, st); break;
    case 24: dslash_bc<T, 24>(g, U, in, out, B, dagger, kappa, st); break;
    case 48: dslash_bc<T, 48>(g, U, in, out, B, dagger, kappa, st); break;
    default: break;
    }
}
template void launch_dslash<double>(const Geom &, const void *, const void *, void *, int, int, int, double,
                                    cudaStream_t);
template void launch_dslash<float>(const Geom &, const void *, const void *, void *, int, int, int, double,
                                   cudaStream_t);

// ------------------------------------------------------------------ allocation-free dslash
// smpq_dslash_noalloc keeps its scratch (the tiled copies of the input and the
// output field that the kernel reads and writes) in this file-scope device
// array instead of asking for device memory.  The array is created when the
// library's device code is loaded on a GPU and stays reserved on every GPU that
// loads the library until the process exits.
#define SMPQ_NOALLOC_SCRATCH_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[SMPQ_NOALLOC_SCRATCH_BYTES];

#include <mutex>

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side handle, so the address is looked up
// once per device (with that device current) and cached.
int noalloc_scratch(smpq_ctx *ctx, int dev, void **out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return set_err(ctx, SMPQ_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_check(ctx, e != cudaSuccess ? e : cudaErrorInvalidSymbol, "scratch address");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SMPQ_OK;
}
} // namespace

extern "C" int smpq_dslash_noalloc(smpq_ctx *ctx, const double *in, double *out, int B, int dagger, int precision) {
    if (!ctx) return SMPQ_EINVAL;
    if (!ctx->have_gauge) return set_err(ctx, SMPQ_ESTATE, "no gauge field loaded");
    if (!in || !out || B < 1) return set_err(ctx, SMPQ_EINVAL, "bad dslash_noalloc arguments");
    if (precision != SMPQ_FP64 && precision != SMPQ_FP32) return set_err(ctx, SMPQ_EINVAL, "bad precision");
    // in and out must be device memory of the context's GPU: a host pointer or
    // another GPU's buffer would be dereferenced by the kernels
    int rc0;
    if ((rc0 = check_device_ptr(ctx, in, "dslash_noalloc in")) || (rc0 = check_device_ptr(ctx, out, "dslash_noalloc out")))
        return rc0;
    const size_t n = (size_t)ctx->V * 12 * B;
    const size_t esz = precision == SMPQ_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t half = ((n * esz + 255) / 256) * 256; // input tile, then output tile
    if (2 * half > SMPQ_NOALLOC_SCRATCH_BYTES)
        return set_err(ctx, SMPQ_EINVAL,
                       "field too large for smpq_dslash_noalloc: needs " + std::to_string(2 * half) +
                           " bytes of scratch, the limit is " + std::to_string(SMPQ_NOALLOC_SCRATCH_BYTES) +
                           " (2 * V * 12 * B * " + std::to_string(esz) + " bytes)");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    void *scratch = nullptr;
    int rc = noalloc_scratch(ctx, ctx->device, &scratch);
    if (rc == SMPQ_OK) {
        cudaStream_t st = ctx->stream;
        if (ctx->user_stream) {
            cudaEventRecord(ctx->ev0, (cudaStream_t)ctx->user_stream);
            cudaStreamWaitEvent(st, ctx->ev0, 0);
        }
        char *tin = (char *)scratch, *tout = (char *)scratch + half;
        const int BC = 1;
        if (precision == SMPQ_FP64) {
            launch_to_tiled<double>(in, tin, ctx->V, B, BC, st);
            launch_dslash<double>(ctx->geom, ctx->U64.p, tin, tout, B, BC, dagger, ctx->opt.kappa, st);
            launch_from_tiled<double>(tout, out, ctx->V, B, BC, st);
        } else {
            launch_to_tiled<float>(in, tin, ctx->V, B, BC, st);
            launch_dslash<float>(ctx->geom, ctx->U32.p, tin, tout, B, BC, dagger, ctx->opt.kappa, st);
            launch_from_tiled<float>(tout, out, ctx->V, B, BC, st);
        }
        cudaError_t e = cudaStreamSynchronize(st);
        rc = e != cudaSuccess ? cuda_check(ctx, e, "dslash_noalloc") : cuda_check(ctx, cudaGetLastError(), "dslash_noalloc launch");
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}
