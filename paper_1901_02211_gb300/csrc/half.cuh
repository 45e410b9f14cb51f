// Half-precision storage formats shared by the stand-alone D_W (half.cu) and
// the solver's half-storage iterations (msolve.cu): FP16 or BF16 complex
// components scaled by one FP32 norm per site and right-hand side, links as
// rows 0 and 1 (reconstruct-12), FP32 arithmetic.  Layout of a field of B
// columns in RHS tiles of BC: components [j / BC][V][12][BC] (one complex
// number as two halves, value = norm * stored), then norms [j / BC][V][BC].
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <string.h>

#include "wilson.cuh"

struct H16 {
    typedef __half2 h2;
    static __device__ __forceinline__ float2 f2(h2 v) { return __half22float2(v); }
    static __device__ __forceinline__ h2 pack(float2 v) { return __float22half2_rn(v); }
};
struct B16 {
    typedef __nv_bfloat162 h2;
    static __device__ __forceinline__ float2 f2(h2 v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ h2 pack(float2 v) { return __float22bfloat162_rn(v); }
};

template <typename HT> __device__ __forceinline__ float2 f2_bits(unsigned w) {
    typename HT::h2 v;
    memcpy(&v, &w, 4);
    return HT::f2(v);
}
template <typename HT> __device__ __forceinline__ unsigned bits_f2(float2 v) {
    typename HT::h2 h = HT::pack(v);
    unsigned w;
    memcpy(&w, &h, 4);
    return w;
}

// NR adjacent columns of one component (NR = 2: one 8-byte access)
template <typename HT, int NR>
__device__ __forceinline__ void ld_cols(const typename HT::h2 *__restrict__ p, float2 v[NR]) {
    if constexpr (NR == 2) {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        v[0] = f2_bits<HT>(q.x);
        v[1] = f2_bits<HT>(q.y);
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = HT::f2(p[r]);
    }
}
template <typename HT, int NR> __device__ __forceinline__ void st_cols(typename HT::h2 *p, const float2 v[NR]) {
    if constexpr (NR == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(bits_f2<HT>(v[0]), bits_f2<HT>(v[1]));
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) p[r] = HT::pack(v[r]);
    }
}
template <int NR> __device__ __forceinline__ void ld_norms(const float *__restrict__ p, float v[NR]) {
    if constexpr (NR == 2) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        v[0] = q.x;
        v[1] = q.y;
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = p[r];
    }
}

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// The link of (mu, s) as a full 3x3 matrix: rows 0 and 1 from memory (24 bytes,
// three 8-byte loads), row 2 = conj(row 0 x row 1).
template <typename HT>
__device__ __forceinline__ void load_link12(const typename HT::h2 *__restrict__ U, size_t idx, float2 m[3][3]) {
    const uint2 *p = reinterpret_cast<const uint2 *>(U + idx * 6);
    const uint2 a = p[0], b = p[1], c = p[2];
    m[0][0] = f2_bits<HT>(a.x);
    m[0][1] = f2_bits<HT>(a.y);
    m[0][2] = f2_bits<HT>(b.x);
    m[1][0] = f2_bits<HT>(b.y);
    m[1][1] = f2_bits<HT>(c.x);
    m[1][2] = f2_bits<HT>(c.y);
    m[2][0] = conjf2(csub(cmul(m[0][1], m[1][2]), cmul(m[0][2], m[1][1])));
    m[2][1] = conjf2(csub(cmul(m[0][2], m[1][0]), cmul(m[0][0], m[1][2])));
    m[2][2] = conjf2(csub(cmul(m[0][0], m[1][1]), cmul(m[0][1], m[1][0])));
}

// One hop, acc += f (1 + SG g_mu) W psi(nb) for NR columns, W = U(ls) or
// U(ls)^dag (BACK); f = the neighbour's norm, negated across an antiperiodic
// boundary (flip).  Same projection as the FP32 hop (S_mu on the lower half).
template <typename HT, int MU, int SG, bool BACK, int BC, int NR>
__device__ __forceinline__ void hop_half(const typename HT::h2 *__restrict__ U, const typename HT::h2 *__restrict__ in,
                                         const float *__restrict__ nrm, int Vl, int nb, int ls, bool flip,
                                         float2 acc[12][NR]) {
    const typename HT::h2 *q = in + (size_t)nb * (12 * BC);
    float f[NR];
    ld_norms<NR>(nrm + (size_t)nb * BC, f);
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (flip) f[r] = -f[r];
    float2 h[2][3][NR];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 p0[NR], p1[NR], p2[NR], p3[NR];
        ld_cols<HT, NR>(q + a * BC, p0);
        ld_cols<HT, NR>(q + (3 + a) * BC, p1);
        ld_cols<HT, NR>(q + (6 + a) * BC, p2);
        ld_cols<HT, NR>(q + (9 + a) * BC, p3);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            float2 s0, s1;
            s_apply<MU>(p2[r], p3[r], s0, s1);
            if (SG > 0) { h[0][a][r] = cadd(p0[r], s0); h[1][a][r] = cadd(p1[r], s1); }
            else { h[0][a][r] = csub(p0[r], s0); h[1][a][r] = csub(p1[r], s1); }
        }
    }
    float2 m[3][3];
    load_link12<HT>(U, (size_t)MU * Vl + ls, m);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (BACK) { // (U^dag)_{ab} = conj(U_{ba})
                    w0 = cfmac(m[b][a], h[0][b][r], w0);
                    w1 = cfmac(m[b][a], h[1][b][r], w1);
                } else {
                    w0 = cfma(m[a][b], h[0][b][r], w0);
                    w1 = cfma(m[a][b], h[1][b][r], w1);
                }
            }
            w0 = cscale(f[r], w0);
            w1 = cscale(f[r], w1);
            acc[a][r] = cadd(acc[a][r], w0);
            acc[3 + a][r] = cadd(acc[3 + a][r], w1);
            float2 l0, l1;
            sdag_apply<MU>(w0, w1, l0, l1);
            if (SG > 0) { acc[6 + a][r] = cadd(acc[6 + a][r], l0); acc[9 + a][r] = cadd(acc[9 + a][r], l1); }
            else { acc[6 + a][r] = csub(acc[6 + a][r], l0); acc[9 + a][r] = csub(acc[9 + a][r], l1); }
        }
    }
}

template <typename HT, int MU, bool DAG, int BC, int NR>
__device__ __forceinline__ void hop_dir_half(const Geom &g, const SiteCoords &xc, const typename HT::h2 *U,
                                             const typename HT::h2 *in, const float *nrm, int s,
                                             float2 acc[12][NR]) {
    const int n = g.n[MU], st = g.stride[MU], c = xc.x[MU];
    const bool top = c == n - 1, bot = c == 0;
    const int nf = top ? s - (n - 1) * st : s + st;
    const int nbk = bot ? s + (n - 1) * st : s - st;
    hop_half<HT, MU, DAG ? +1 : -1, false, BC, NR>(U, in, nrm, g.V, nf, s, top && g.bcf[MU] < 0, acc);
    hop_half<HT, MU, DAG ? -1 : +1, true, BC, NR>(U, in, nrm, g.V, nbk, nbk, bot && g.bcf[MU] < 0, acc);
}

// acc = hop(s) for one column of a half-format field (`in` and `nrm` already
// offset by tile and column)
template <typename HT, bool DAG, int BC>
__device__ __forceinline__ void wilson_hop_half(const Geom &g, const typename HT::h2 *__restrict__ U,
                                                const typename HT::h2 *__restrict__ in, const float *__restrict__ nrm,
                                                int s, float2 acc[12][1]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c][0] = make_float2(0.f, 0.f);
    const SiteCoords xc(g, s);
    hop_dir_half<HT, 0, DAG, BC, 1>(g, xc, U, in, nrm, s, acc);
    hop_dir_half<HT, 1, DAG, BC, 1>(g, xc, U, in, nrm, s, acc);
    hop_dir_half<HT, 2, DAG, BC, 1>(g, xc, U, in, nrm, s, acc);
    hop_dir_half<HT, 3, DAG, BC, 1>(g, xc, U, in, nrm, s, acc);
}

// the 12 components of one column at one site: v = norm * stored value
template <typename HT, int BC>
__device__ __forceinline__ void ld_site_half(const typename HT::h2 *__restrict__ q, float n, float2 v[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const float2 f = HT::f2(q[c * BC]);
        v[c] = make_float2(n * f.x, n * f.y);
    }
}
// store the 12 components of one column at one site with their norm
// (largest |re|, |im|); returns the norm
template <typename HT, int BC>
__device__ __forceinline__ float st_site_half(typename HT::h2 *__restrict__ q, float *__restrict__ nrm,
                                              const float2 v[12]) {
    float mx = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) mx = fmaxf(mx, fmaxf(fabsf(v[c].x), fabsf(v[c].y)));
    // below the smallest normal FP32 number the reciprocal would overflow:
    // such a site is stored as zero
    const bool tiny = !(mx >= 1.17549435e-38f);
    const float inv = tiny ? 0.f : 1.f / mx;
#pragma unroll
    for (int c = 0; c < 12; ++c) q[c * BC] = HT::pack(make_float2(inv * v[c].x, inv * v[c].y));
    *nrm = tiny ? 0.f : mx;
    return mx;
}

// ---------------------------------------------------------------- two columns in packed lanes
// Two adjacent right-hand-side columns per thread, held as the two lanes of
// packed FP32 instructions (FFMA2, FADD2, FMUL2 on sm_100 and later): every
// complex value is a pair of float2, .r = (re col 0, re col 1) and .i = (im
// col 0, im col 1).  Each arithmetic instruction then serves both columns, and
// a link (loaded and reconstructed once) serves both.
struct c2 {
    float2 r, i;
};
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

template <typename HT> __device__ __forceinline__ c2 ld_c2(const typename HT::h2 *__restrict__ p) {
    const uint2 q = *reinterpret_cast<const uint2 *>(p);
    const float2 a = f2_bits<HT>(q.x), b = f2_bits<HT>(q.y);
    return {make_float2(a.x, b.x), make_float2(a.y, b.y)};
}
template <typename HT> __device__ __forceinline__ void st_c2(typename HT::h2 *p, float2 r, float2 i) {
    *reinterpret_cast<uint2 *>(p) =
        make_uint2(bits_f2<HT>(make_float2(r.x, i.x)), bits_f2<HT>(make_float2(r.y, i.y)));
}

// a + g * u * v for a unit u: K = 0: 1, 1: -1, 2: i, 3: -i
template <int K> __device__ __forceinline__ c2 fma_unit(float g, c2 v, c2 a) {
    if (K == 0) return {__ffma2_rn(bc2(g), v.r, a.r), __ffma2_rn(bc2(g), v.i, a.i)};
    if (K == 1) return {__ffma2_rn(bc2(-g), v.r, a.r), __ffma2_rn(bc2(-g), v.i, a.i)};
    if (K == 2) return {__ffma2_rn(bc2(-g), v.i, a.r), __ffma2_rn(bc2(g), v.r, a.i)};
    return {__ffma2_rn(bc2(g), v.i, a.r), __ffma2_rn(bc2(-g), v.r, a.i)};
}
// S_mu (l0, l1) = (u0 l_{J0}, u1 l_{J1}) and S_mu^dag (w0, w1) = (v0 w_{D0}, v1 w_{D1});
// unit codes as in fma_unit
template <int MU> struct SPerm {
    static constexpr int J0 = (MU == 0 || MU == 1) ? 1 : 0, J1 = 1 - J0;
    static constexpr int U0 = MU == 0 ? 3 : MU == 1 ? 1 : MU == 2 ? 3 : 0;
    static constexpr int U1 = MU == 0 ? 3 : MU == 1 ? 0 : MU == 2 ? 2 : 0;
    static constexpr int D0 = J0, D1 = J1;
    static constexpr int V0 = MU == 0 ? 2 : MU == 1 ? 0 : MU == 2 ? 2 : 0;
    static constexpr int V1 = MU == 0 ? 2 : MU == 1 ? 1 : MU == 2 ? 3 : 0;
};

template <typename HT, int MU, int SG, bool BACK, int BC>
__device__ __forceinline__ void hop_half_c2(const typename HT::h2 *__restrict__ U, const typename HT::h2 *__restrict__ in,
                                            const float *__restrict__ nrm, int Vl, int nb, int ls, bool flip,
                                            c2 acc[12]) {
    typedef SPerm<MU> P;
    const typename HT::h2 *q = in + (size_t)nb * (12 * BC);
    float2 f = *reinterpret_cast<const float2 *>(nrm + (size_t)nb * BC);
    if (flip) f = make_float2(-f.x, -f.y);
    const float g = (float)SG;
    c2 h0[3], h1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const c2 p0 = ld_c2<HT>(q + a * BC), p1 = ld_c2<HT>(q + (3 + a) * BC);
        const c2 p2 = ld_c2<HT>(q + (6 + a) * BC), p3 = ld_c2<HT>(q + (9 + a) * BC);
        h0[a] = fma_unit<P::U0>(g, P::J0 ? p3 : p2, p0);
        h1[a] = fma_unit<P::U1>(g, P::J1 ? p3 : p2, p1);
    }
    float2 m[3][3];
    load_link12<HT>(U, (size_t)MU * Vl + ls, m);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c2 w0 = {bc2(0.f), bc2(0.f)}, w1 = w0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float2 e = BACK ? m[b][a] : m[a][b]; // W_ab = conj(U_ba) for BACK
            const float2 ex = bc2(e.x), ey = bc2(BACK ? -e.y : e.y), ney = bc2(BACK ? e.y : -e.y);
            w0.r = __ffma2_rn(ex, h0[b].r, __ffma2_rn(ney, h0[b].i, w0.r));
            w0.i = __ffma2_rn(ex, h0[b].i, __ffma2_rn(ey, h0[b].r, w0.i));
            w1.r = __ffma2_rn(ex, h1[b].r, __ffma2_rn(ney, h1[b].i, w1.r));
            w1.i = __ffma2_rn(ex, h1[b].i, __ffma2_rn(ey, h1[b].r, w1.i));
        }
        w0 = {__fmul2_rn(f, w0.r), __fmul2_rn(f, w0.i)};
        w1 = {__fmul2_rn(f, w1.r), __fmul2_rn(f, w1.i)};
        acc[a] = {__fadd2_rn(acc[a].r, w0.r), __fadd2_rn(acc[a].i, w0.i)};
        acc[3 + a] = {__fadd2_rn(acc[3 + a].r, w1.r), __fadd2_rn(acc[3 + a].i, w1.i)};
        acc[6 + a] = fma_unit<P::V0>(g, P::D0 ? w1 : w0, acc[6 + a]);
        acc[9 + a] = fma_unit<P::V1>(g, P::D1 ? w1 : w0, acc[9 + a]);
    }
}

template <typename HT, int MU, bool DAG, int BC>
__device__ __forceinline__ void hop_dir_half_c2(const Geom &g, const SiteCoords &xc, const typename HT::h2 *U,
                                                const typename HT::h2 *in, const float *nrm, int s, c2 acc[12]) {
    const int n = g.n[MU], st = g.stride[MU], c = xc.x[MU];
    const bool top = c == n - 1, bot = c == 0;
    const int nf = top ? s - (n - 1) * st : s + st;
    const int nbk = bot ? s + (n - 1) * st : s - st;
    hop_half_c2<HT, MU, DAG ? +1 : -1, false, BC>(U, in, nrm, g.V, nf, s, top && g.bcf[MU] < 0, acc);
    hop_half_c2<HT, MU, DAG ? -1 : +1, true, BC>(U, in, nrm, g.V, nbk, nbk, bot && g.bcf[MU] < 0, acc);
}

// acc = hop(s) for two columns (packed lanes) of a half-format field
template <typename HT, bool DAG, int BC>
__device__ __forceinline__ void wilson_hop_half_c2(const Geom &g, const typename HT::h2 *__restrict__ U,
                                                   const typename HT::h2 *__restrict__ in,
                                                   const float *__restrict__ nrm, int s, c2 acc[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = {bc2(0.f), bc2(0.f)};
    const SiteCoords xc(g, s);
    hop_dir_half_c2<HT, 0, DAG, BC>(g, xc, U, in, nrm, s, acc);
    hop_dir_half_c2<HT, 1, DAG, BC>(g, xc, U, in, nrm, s, acc);
    hop_dir_half_c2<HT, 2, DAG, BC>(g, xc, U, in, nrm, s, acc);
    hop_dir_half_c2<HT, 3, DAG, BC>(g, xc, U, in, nrm, s, acc);
}

// store the 12 components of two columns at one site (packed lanes) with
// their norms; sites below the smallest normal FP32 number are stored as zero
template <typename HT, int BC>
__device__ __forceinline__ void st_site_half_c2(typename HT::h2 *__restrict__ q, float *__restrict__ nrm,
                                                const c2 v[12]) {
    float mx0 = 0.f, mx1 = 0.f;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        mx0 = fmaxf(mx0, fmaxf(fabsf(v[c].r.x), fabsf(v[c].i.x)));
        mx1 = fmaxf(mx1, fmaxf(fabsf(v[c].r.y), fabsf(v[c].i.y)));
    }
    if (!(mx0 >= 1.17549435e-38f)) mx0 = 0.f;
    if (!(mx1 >= 1.17549435e-38f)) mx1 = 0.f;
    const float2 inv = make_float2(mx0 > 0.f ? 1.f / mx0 : 0.f, mx1 > 0.f ? 1.f / mx1 : 0.f);
#pragma unroll
    for (int c = 0; c < 12; ++c) st_c2<HT>(q + c * BC, __fmul2_rn(inv, v[c].r), __fmul2_rn(inv, v[c].i));
    *reinterpret_cast<float2 *>(nrm) = make_float2(mx0, mx1);
}
