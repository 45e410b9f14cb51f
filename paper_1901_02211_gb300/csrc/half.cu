// Half-precision storage for the stand-alone Wilson dslash D_W (Sec. 2.1,
// around Eq. 3):
//   - spinor components in FP16 or BF16, scaled by one FP32 norm per site and
//     right-hand side (the largest |re| or |im| of its 12 components), so the
//     stored values lie in [-1, 1];
//   - links stored as their first two rows (reconstruct-12): for U in SU(3)
//     the third row is the complex conjugate of the cross product of the
//     first two, recomputed in FP32 at every use;
//   - arithmetic and accumulation in FP32.
// This file holds the stand-alone D_W of smpq_dslash and smpq_time_dslash; the
// solver's half-storage iterations (msolve.cu) share the device code in
// half.cuh.
//
// Layouts (RHS tiles of BC columns, as the FP32 and FP64 fields):
//   components [j / BC][V][12][BC] of H2 (one complex number as two halves)
//   norms      [j / BC][V][BC] float; component value = norm * stored value
//   links      [(mu * V + s) * 6 + row * 3 + col], rows 0 and 1
#include "smpq_internal.cuh"
#include "half.cuh"

// out = D_W in (DAG: D_W^dag), both in the half format; the output norm is
// taken from the FP32 result before it is rounded to the half format.
// (one column per thread fits 80 registers, three 256-thread blocks per SM;
// the two-column form of this scalar kernel is held to two blocks per SM)
template <typename HT, bool DAG, int BC, int NR>
__global__ void __launch_bounds__(TileMap<BC, NR>::THREADS, NR == 1 ? 3 : 2)
    dslash_half_kernel(Geom g, const typename HT::h2 *__restrict__ U, const typename HT::h2 *__restrict__ in,
                       const float *__restrict__ nin, typename HT::h2 *__restrict__ out, float *__restrict__ nout,
                       float kappa) {
    typedef TileMap<BC, NR> TM;
    const int s = blockIdx.x * TM::SPB + threadIdx.x / TM::TPS;
    const int jj = (threadIdx.x % TM::TPS) * NR;
    if (s >= g.V) return;
    const size_t fb = (size_t)blockIdx.y * 12 * g.V * BC + jj, nbase = (size_t)blockIdx.y * g.V * BC + jj;
    const typename HT::h2 *pin = in + fb;
    const float *pn = nin + nbase;
    float2 acc[12][NR];
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[c][r] = make_float2(0.f, 0.f);
    const SiteCoords xc(g, s);
    hop_dir_half<HT, 0, DAG, BC, NR>(g, xc, U, pin, pn, s, acc);
    hop_dir_half<HT, 1, DAG, BC, NR>(g, xc, U, pin, pn, s, acc);
    hop_dir_half<HT, 2, DAG, BC, NR>(g, xc, U, pin, pn, s, acc);
    hop_dir_half<HT, 3, DAG, BC, NR>(g, xc, U, pin, pn, s, acc);
    float ns[NR], mx[NR];
    ld_norms<NR>(pn + (size_t)s * BC, ns);
#pragma unroll
    for (int r = 0; r < NR; ++r) mx[r] = 0.f;
    const typename HT::h2 *ps = pin + (size_t)s * 12 * BC;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        float2 v[NR];
        ld_cols<HT, NR>(ps + c * BC, v);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            float2 o;
            o.x = fmaf(ns[r], v[r].x, -kappa * acc[c][r].x);
            o.y = fmaf(ns[r], v[r].y, -kappa * acc[c][r].y);
            acc[c][r] = o;
            mx[r] = fmaxf(mx[r], fmaxf(fabsf(o.x), fabsf(o.y)));
        }
    }
    float inv[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) { // below the smallest normal FP32 number: stored as zero
        const bool tiny = !(mx[r] >= 1.17549435e-38f);
        inv[r] = tiny ? 0.f : 1.f / mx[r];
        if (tiny) mx[r] = 0.f;
    }
    typename HT::h2 *po = out + fb + (size_t)s * 12 * BC;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        float2 v[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = cscale(inv[r], acc[c][r]);
        st_cols<HT, NR>(po + c * BC, v);
    }
    float *pno = nout + nbase + (size_t)s * BC;
    if constexpr (NR == 2) *reinterpret_cast<float2 *>(pno) = make_float2(mx[0], mx[1]);
    else
#pragma unroll
        for (int r = 0; r < NR; ++r) pno[r] = mx[r];
}

// out = D_W in for two columns per thread (BC even), packed lanes
template <typename HT, bool DAG, int BC>
__global__ void __launch_bounds__(TileMap<BC, 2>::THREADS, 2)
    dslash_half_c2_kernel(Geom g, const typename HT::h2 *__restrict__ U, const typename HT::h2 *__restrict__ in,
                          const float *__restrict__ nin, typename HT::h2 *__restrict__ out, float *__restrict__ nout,
                          float kappa) {
    typedef TileMap<BC, 2> TM;
    const int s = blockIdx.x * TM::SPB + threadIdx.x / TM::TPS;
    const int jj = (threadIdx.x % TM::TPS) * 2;
    if (s >= g.V) return;
    const size_t fb = (size_t)blockIdx.y * 12 * g.V * BC + jj, nbase = (size_t)blockIdx.y * g.V * BC + jj;
    const typename HT::h2 *pin = in + fb;
    const float *pn = nin + nbase;
    c2 acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = {bc2(0.f), bc2(0.f)};
    const SiteCoords xc(g, s);
    hop_dir_half_c2<HT, 0, DAG, BC>(g, xc, U, pin, pn, s, acc);
    hop_dir_half_c2<HT, 1, DAG, BC>(g, xc, U, pin, pn, s, acc);
    hop_dir_half_c2<HT, 2, DAG, BC>(g, xc, U, pin, pn, s, acc);
    hop_dir_half_c2<HT, 3, DAG, BC>(g, xc, U, pin, pn, s, acc);
    const float2 ns = *reinterpret_cast<const float2 *>(pn + (size_t)s * BC), nk = bc2(-kappa);
    float mx0 = 0.f, mx1 = 0.f;
    const typename HT::h2 *ps = pin + (size_t)s * 12 * BC;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const c2 v = ld_c2<HT>(ps + c * BC);
        acc[c].r = __ffma2_rn(ns, v.r, __fmul2_rn(nk, acc[c].r));
        acc[c].i = __ffma2_rn(ns, v.i, __fmul2_rn(nk, acc[c].i));
        mx0 = fmaxf(mx0, fmaxf(fabsf(acc[c].r.x), fabsf(acc[c].i.x)));
        mx1 = fmaxf(mx1, fmaxf(fabsf(acc[c].r.y), fabsf(acc[c].i.y)));
    }
    // below the smallest normal FP32 number the reciprocal would overflow: stored as zero
    if (!(mx0 >= 1.17549435e-38f)) mx0 = 0.f;
    if (!(mx1 >= 1.17549435e-38f)) mx1 = 0.f;
    const float2 inv = make_float2(mx0 > 0.f ? 1.f / mx0 : 0.f, mx1 > 0.f ? 1.f / mx1 : 0.f);
    typename HT::h2 *po = out + fb + (size_t)s * 12 * BC;
#pragma unroll
    for (int c = 0; c < 12; ++c) st_c2<HT>(po + c * BC, __fmul2_rn(inv, acc[c].r), __fmul2_rn(inv, acc[c].i));
    *reinterpret_cast<float2 *>(nout + nbase + (size_t)s * BC) = make_float2(mx0, mx1);
}

// ------------------------------------------------------------------ packing and conversion
// U_aos double[V][4][3][3][2] -> rows 0 and 1 of every link, FP16 and BF16
__global__ void pack_links12_kernel(const double2 *__restrict__ Uaos, __half2 *__restrict__ Uh,
                                    __nv_bfloat162 *__restrict__ Ub, int V) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)V * 24) return;
    const int s = (int)(i / 24), k = (int)(i % 24), mu = k / 6, e = k % 6; // e = row * 3 + col, row < 2
    const double2 u = Uaos[(size_t)s * 36 + mu * 9 + e];
    const float2 f = make_float2((float)u.x, (float)u.y);
    const size_t o = ((size_t)mu * V + s) * 6 + e;
    Uh[o] = H16::pack(f);
    Ub[o] = B16::pack(f);
}

void launch_pack_links12(const double *U_aos, void *Uh, void *Ub, int V, cudaStream_t st) {
    const long n = (long)V * 24;
    pack_links12_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double2 *)U_aos, (__half2 *)Uh,
                                                                      (__nv_bfloat162 *)Ub, V);
}

// ABI double[V][12][B][2] -> half format (tile BC); one thread per (site, rhs).
// norm = FP32 copy of max |re|, |im|; stored value = component / norm.
template <typename HT>
__global__ void to_half_kernel(const double2 *__restrict__ in, typename HT::h2 *__restrict__ out,
                               float *__restrict__ nout, int V, int B, int BC) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)V * B) return;
    const int j = (int)(i % B), s = (int)(i / B);
    double2 v[12];
    double mx = 0;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        v[c] = in[((size_t)s * 12 + c) * B + j];
        mx = fmax(mx, fmax(fabs(v[c].x), fabs(v[c].y)));
    }
    const float n = (float)mx;
    const double dn = n > 0.f ? (double)n : 1.0;
    const size_t t = (size_t)(j / BC), jj = (size_t)(j % BC);
#pragma unroll
    for (int c = 0; c < 12; ++c)
        out[((t * V + s) * 12 + c) * BC + jj] = HT::pack(make_float2((float)(v[c].x / dn), (float)(v[c].y / dn)));
    nout[(t * V + s) * BC + jj] = n;
}

template <typename HT>
__global__ void from_half_kernel(const typename HT::h2 *__restrict__ in, const float *__restrict__ nin,
                                 double2 *__restrict__ out, int V, int B, int BC) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)V * B) return;
    const int j = (int)(i % B), s = (int)(i / B);
    const size_t t = (size_t)(j / BC), jj = (size_t)(j % BC);
    const double n = nin[(t * V + s) * BC + jj];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const float2 f = HT::f2(in[((t * V + s) * 12 + c) * BC + jj]);
        out[((size_t)s * 12 + c) * B + j] = make_double2(n * (double)f.x, n * (double)f.y);
    }
}

// ------------------------------------------------------------------ launchers
// Tile width of the half-format fields for B columns: 16-column tiles (a
// site's component is 64 contiguous bytes) when B allows, else one column.
int half_tile(int B) { return B % 16 == 0 ? 16 : 1; }

// columns per thread in 16-column tiles: 2 = dslash_half_c2_kernel (packed
// lanes, 8-byte accesses, 128 registers), 1 = dslash_half_kernel (80
// registers).  On the 8^3x16 lattice with 3072 columns: 1.37 / 1.33 ms per
// FP16 / BF16 launch with 2, 1.58 / 1.73 ms with 1.
#ifndef SMPQ_HALF_NR
#define SMPQ_HALF_NR 2
#endif

size_t half_field_bytes(int V, int B) { return (size_t)V * B * (12 * 4) + (size_t)V * B * 4; }

template <typename HT, int BC, int NR>
static void dslash_half_bc(const Geom &g, const void *U, const void *in, void *out, int B, int dagger, float kappa,
                           cudaStream_t st) {
    typedef typename HT::h2 h2;
    typedef TileMap<BC, NR> TM;
    const size_t ncomp = (size_t)g.V * 12 * B;
    const h2 *pin = (const h2 *)in;
    const float *nin = (const float *)(pin + ncomp);
    h2 *pout = (h2 *)out;
    float *nout = (float *)(pout + ncomp);
    const dim3 grid((g.V + TM::SPB - 1) / TM::SPB, B / BC);
    if constexpr (NR == 2) {
        if (dagger)
            dslash_half_c2_kernel<HT, true, BC><<<grid, TM::THREADS, 0, st>>>(g, (const h2 *)U, pin, nin, pout, nout,
                                                                              kappa);
        else
            dslash_half_c2_kernel<HT, false, BC><<<grid, TM::THREADS, 0, st>>>(g, (const h2 *)U, pin, nin, pout,
                                                                               nout, kappa);
    } else {
        if (dagger)
            dslash_half_kernel<HT, true, BC, NR><<<grid, TM::THREADS, 0, st>>>(g, (const h2 *)U, pin, nin, pout,
                                                                               nout, kappa);
        else
            dslash_half_kernel<HT, false, BC, NR><<<grid, TM::THREADS, 0, st>>>(g, (const h2 *)U, pin, nin, pout,
                                                                                nout, kappa);
    }
}

// A half-format field of B columns is one buffer: the V * 12 * B components
// (tile layout) followed by the V * B norms.
template <typename HT>
static void dslash_half_t(const Geom &g, const void *U, const void *in, void *out, int B, int dagger, double kappa,
                          cudaStream_t st) {
    switch (half_tile(B)) {
    case 16: dslash_half_bc<HT, 16, SMPQ_HALF_NR>(g, U, in, out, B, dagger, (float)kappa, st); break;
    default: dslash_half_bc<HT, 1, 1>(g, U, in, out, B, dagger, (float)kappa, st); break;
    }
}

void launch_dslash_half(int prec, const Geom &g, const void *U, const void *in, void *out, int B, int dagger,
                        double kappa, cudaStream_t st) {
    if (prec == SMPQ_BF16N) dslash_half_t<B16>(g, U, in, out, B, dagger, kappa, st);
    else dslash_half_t<H16>(g, U, in, out, B, dagger, kappa, st);
}

void launch_to_half(int prec, const double *in, void *out, int V, int B, cudaStream_t st) {
    const long n = (long)V * B;
    const unsigned nb = (unsigned)((n + 255) / 256);
    const int BC = half_tile(B);
    const size_t ncomp = (size_t)V * 12 * B;
    if (prec == SMPQ_BF16N) {
        __nv_bfloat162 *o = (__nv_bfloat162 *)out;
        to_half_kernel<B16><<<nb, 256, 0, st>>>((const double2 *)in, o, (float *)(o + ncomp), V, B, BC);
    } else {
        __half2 *o = (__half2 *)out;
        to_half_kernel<H16><<<nb, 256, 0, st>>>((const double2 *)in, o, (float *)(o + ncomp), V, B, BC);
    }
}

void launch_from_half(int prec, const void *in, double *out, int V, int B, cudaStream_t st) {
    const long n = (long)V * B;
    const unsigned nb = (unsigned)((n + 255) / 256);
    const int BC = half_tile(B);
    const size_t ncomp = (size_t)V * 12 * B;
    if (prec == SMPQ_BF16N) {
        const __nv_bfloat162 *p = (const __nv_bfloat162 *)in;
        from_half_kernel<B16><<<nb, 256, 0, st>>>(p, (const float *)(p + ncomp), (double2 *)out, V, B, BC);
    } else {
        const __half2 *p = (const __half2 *)in;
        from_half_kernel<H16><<<nb, 256, 0, st>>>(p, (const float *)(p + ncomp), (double2 *)out, V, B, BC);
    }
}
