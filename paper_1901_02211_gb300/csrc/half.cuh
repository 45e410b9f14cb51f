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
