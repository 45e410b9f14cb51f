// Wilson hopping term of D_W (Sec. 2.1, around Eq. 3) for one site and NR
// right-hand sides, with half-spinor projection.
//
//   hop(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
//   D_W psi(x) = psi(x) - kappa hop(x)
// With DAG = true the projector signs are exchanged, which gives
// gamma_5 D_W gamma_5 = D_W^dag (so H^2 = D_W^dag D_W needs no explicit gamma_5).
//
// Chiral basis: g_mu = [[0, S_mu], [S_mu^dag, 0]] with S_k = -i sigma_k (k = x, y, z)
// and S_t = 1.  (1 + s g_mu) psi has upper half h = psi_up + s S_mu psi_lo and
// lower half s S_mu^dag h, so only h (2 spins x 3 colours) is multiplied by the
// link: 2 colour mat-vecs per hop instead of 4.
//
// A thread handles NR adjacent right-hand-side columns of one site: the link
// and the neighbour index are fetched once for all NR columns, and two FP32
// columns move as one 16-byte access.
#pragma once
#include <type_traits>

#include "device.cuh"

// S_mu l  for the lower 2-spinor l = (l0, l1)
template <int MU, typename C> __device__ __forceinline__ void s_apply(C l0, C l1, C &o0, C &o1) {
    if (MU == 0) { o0 = cneg(cmuli(l1)); o1 = cneg(cmuli(l0)); }        // -i sigma_x
    else if (MU == 1) { o0 = cneg(l1); o1 = l0; }                       // -i sigma_y
    else if (MU == 2) { o0 = cneg(cmuli(l0)); o1 = cmuli(l1); }         // -i sigma_z
    else { o0 = l0; o1 = l1; }                                          // 1
}
// S_mu^dag u
template <int MU, typename C> __device__ __forceinline__ void sdag_apply(C u0, C u1, C &o0, C &o1) {
    if (MU == 0) { o0 = cmuli(u1); o1 = cmuli(u0); }
    else if (MU == 1) { o0 = u1; o1 = cneg(u0); }
    else if (MU == 2) { o0 = cmuli(u0); o1 = cneg(cmuli(u1)); }
    else { o0 = u0; o1 = u1; }
}

// NR adjacent complex values, with one access where the width allows it
template <typename C, int NR> struct Cols {
    static __device__ __forceinline__ void load(const C *p, C v[NR]) {
#pragma unroll
        for (int r = 0; r < NR; ++r) v[r] = p[r];
    }
    static __device__ __forceinline__ void store(C *p, const C v[NR]) {
#pragma unroll
        for (int r = 0; r < NR; ++r) p[r] = v[r];
    }
};
template <> struct Cols<float2, 2> {
    static __device__ __forceinline__ void load(const float2 *p, float2 v[2]) {
        float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = make_float2(q.x, q.y);
        v[1] = make_float2(q.z, q.w);
    }
    static __device__ __forceinline__ void store(float2 *p, const float2 v[2]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    }
};

// One hop: acc += (1 + SG g_mu) W psi(nb) * f for NR columns, with W = U
// (BACK = false) or U^dag (BACK = true) read from link site ls; the boundary
// factor f is +1 or -1 and enters as a sign (flip = f < 0).
// `in` points at the tile (plus first column): site nb starts at nb * 12 * BC;
// links U[(MU * Vl + ls) * 9 + e].  (Vf, the field site count, is not needed.)
template <typename T, int MU, int SG, bool BACK, int BC, int NR = 1>
__device__ __forceinline__ void hop_one(const typename cplx_t<T>::type *__restrict__ U,
                                        const typename cplx_t<T>::type *__restrict__ in, int Vf, int Vl, int nb,
                                        int ls, bool flip, typename cplx_t<T>::type acc[12][NR]) {
    typedef typename cplx_t<T>::type C;
    const C *q = in + (size_t)nb * (12 * BC); // the 12 components of a site are BC apart
    // project colour by colour: only the 4 spin components of one colour are live
    C h[2][3][NR];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        C p0[NR], p1[NR], p2[NR], p3[NR];
        Cols<C, NR>::load(q + a * BC, p0);
        Cols<C, NR>::load(q + (3 + a) * BC, p1);
        Cols<C, NR>::load(q + (6 + a) * BC, p2);
        Cols<C, NR>::load(q + (9 + a) * BC, p3);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            C s0, s1;
            s_apply<MU>(p2[r], p3[r], s0, s1);
            if (SG > 0) { h[0][a][r] = cadd(p0[r], s0); h[1][a][r] = cadd(p1[r], s1); }
            else { h[0][a][r] = csub(p0[r], s0); h[1][a][r] = csub(p1[r], s1); }
        }
    }
    // colour multiply and reconstruct one colour row at a time: only one row
    // (or column, for U^dag) of the link is live
    const C *ul = U + ((size_t)MU * Vl + ls) * 9; // the 9 elements of a link are contiguous
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        C ur[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) ur[b] = BACK ? ul[b * 3 + a] : ul[a * 3 + b];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            C w0 = mkc<C>(0, 0), w1 = mkc<C>(0, 0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (BACK) {
                    w0 = cfmac(ur[b], h[0][b][r], w0);
                    w1 = cfmac(ur[b], h[1][b][r], w1);
                } else {
                    w0 = cfma(ur[b], h[0][b][r], w0);
                    w1 = cfma(ur[b], h[1][b][r], w1);
                }
            }
            if (flip) {
                w0 = cneg(w0);
                w1 = cneg(w1);
            }
            acc[a][r] = cadd(acc[a][r], w0);
            acc[3 + a][r] = cadd(acc[3 + a][r], w1);
            C l0, l1;
            sdag_apply<MU>(w0, w1, l0, l1);
            if (SG > 0) { acc[6 + a][r] = cadd(acc[6 + a][r], l0); acc[9 + a][r] = cadd(acc[9 + a][r], l1); }
            else { acc[6 + a][r] = csub(acc[6 + a][r], l0); acc[9 + a][r] = csub(acc[9 + a][r], l1); }
        }
    }
}

// SMPQ_HOP_FENCE: a compiler-only memory fence between hops, so the loads of
// later hops are not hoisted above earlier ones (bounds the live registers).
// It emits no instruction and never waits.
#ifdef SMPQ_HOP_FENCE
#define SMPQ_HOP_BARRIER() asm volatile("" ::: "memory")
#else
#define SMPQ_HOP_BARRIER()
#endif

// Lattice coordinates of site s (three integer divisions, once per site).
struct SiteCoords {
    int x[4];
    __device__ __forceinline__ SiteCoords(const Geom &g, int s) {
        int r = s;
        x[0] = r % g.n[0];
        r /= g.n[0];
        x[1] = r % g.n[1];
        r /= g.n[1];
        x[2] = r % g.n[2];
        x[3] = r / g.n[2];
    }
};

template <typename T, int MU, bool DAG, int BC, int NR>
__device__ __forceinline__ void hop_dir(const Geom &g, const SiteCoords &xc,
                                        const typename cplx_t<T>::type *__restrict__ U,
                                        const typename cplx_t<T>::type *__restrict__ in, int s,
                                        typename cplx_t<T>::type acc[12][NR]) {
    const int n = g.n[MU], st = g.stride[MU], c = xc.x[MU];
    const bool top = c == n - 1, bot = c == 0;
    const int nf = top ? s - (n - 1) * st : s + st;
    const int nbk = bot ? s + (n - 1) * st : s - st;
    const bool ff = top && g.bcf[MU] < 0;
    const bool fb = bot && g.bcf[MU] < 0;
    // forward: (1 - g) U(x) psi(x+mu)   [DAG: (1 + g)]
    hop_one<T, MU, DAG ? +1 : -1, false, BC, NR>(U, in, g.V, g.V, nf, s, ff, acc);
    SMPQ_HOP_BARRIER();
    // backward: (1 + g) U(x-mu)^dag psi(x-mu)   [DAG: (1 - g)]
    hop_one<T, MU, DAG ? -1 : +1, true, BC, NR>(U, in, g.V, g.V, nbk, nbk, fb, acc);
    SMPQ_HOP_BARRIER();
}

// acc = hop(s) for the NR columns whose tile base pointer is `in`
// (already offset by tile and first column).
template <typename T, bool DAG, int BC, int NR = 1>
__device__ __forceinline__ void wilson_hop(const Geom &g, const typename cplx_t<T>::type *__restrict__ U,
                                           const typename cplx_t<T>::type *__restrict__ in, int s,
                                           typename cplx_t<T>::type acc[12][NR]) {
    typedef typename cplx_t<T>::type C;
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[c][r] = mkc<C>(0, 0);
    const SiteCoords xc(g, s);
    hop_dir<T, 0, DAG, BC, NR>(g, xc, U, in, s, acc);
    hop_dir<T, 1, DAG, BC, NR>(g, xc, U, in, s, acc);
    hop_dir<T, 2, DAG, BC, NR>(g, xc, U, in, s, acc);
    hop_dir<T, 3, DAG, BC, NR>(g, xc, U, in, s, acc);
}

// ---------------------------------------------------------------- rolled variant
// The same hop as one loop over the 8 (direction, orientation) pairs, for the
// float-float kernels: their unrolled code overflows the instruction cache
// (ncu: "no instruction" the leading stall).  S_mu and S_mu^dag are
// unit-modulus permutations applied with selects, the projector sign and the
// link orientation are runtime values.

// c * v for c in {1, -1, i, -i}: rot = multiply by i, neg = negate
template <typename C> __device__ __forceinline__ C unit_mul(C v, bool rot, bool neg) {
    C r = rot ? cmuli(v) : v;
    return neg ? cneg(r) : r;
}
// S_mu l: mu 0: (-i l1, -i l0); 1: (-l1, l0); 2: (-i l0, i l1); 3: (l0, l1)
template <typename C> __device__ __forceinline__ void s_apply_rt(int mu, C l0, C l1, C &o0, C &o1) {
    const bool sw = mu <= 1;
    C a = sw ? l1 : l0, b = sw ? l0 : l1;
    o0 = unit_mul(a, mu == 0 || mu == 2, mu <= 2);
    o1 = unit_mul(b, mu == 0 || mu == 2, mu == 0);
}
// S_mu^dag u: mu 0: (i u1, i u0); 1: (u1, -u0); 2: (i u0, -i u1); 3: (u0, u1)
template <typename C> __device__ __forceinline__ void sdag_apply_rt(int mu, C u0, C u1, C &o0, C &o1) {
    const bool sw = mu <= 1;
    C a = sw ? u1 : u0, b = sw ? u0 : u1;
    o0 = unit_mul(a, mu == 0 || mu == 2, false);
    o1 = unit_mul(b, mu == 0 || mu == 2, mu == 1 || mu == 2);
}

// Float-float sums inside the hop are left unnormalised (cadd_lazy, cdot3_lazy)
// and the 12 accumulators are renormalised once after the 8 hops;
// SMPQ_DF64_EAGER renormalises after every operation instead.  (The default
// float-float path is hop_one_pairs below; this generic one serves it with
// SMPQ_DF64_UNPAIRED or SMPQ_DF64_EAGER, and FP32 with SMPQ_FP32_ROLLED.)
#ifdef SMPQ_DF64_EAGER
#define SMPQ_HADD cadd
#define SMPQ_HDOT cdot3
#else
#define SMPQ_HADD cadd_lazy
#define SMPQ_HDOT cdot3_lazy
#endif

// U^dag is read as the transpose of U with conjugated elements (back = true).
template <typename C> __device__ __forceinline__ C conj_if(C v, bool c) {
    C r = v;
    if (c) r.y = -r.y;
    return r;
}
template <typename T, int BC, int NR>
__device__ __forceinline__ void hop_one_rt(int mu, bool plus, bool back, const typename cplx_t<T>::type *__restrict__ U,
                                           const typename cplx_t<T>::type *__restrict__ in, int Vl, int nb, int ls,
                                           bool flip, typename cplx_t<T>::type acc[12][NR]) {
    typedef typename cplx_t<T>::type C;
    const C *q = in + (size_t)nb * (12 * BC);
    C h[2][3][NR];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        C p0[NR], p1[NR], p2[NR], p3[NR];
        Cols<C, NR>::load(q + a * BC, p0);
        Cols<C, NR>::load(q + (3 + a) * BC, p1);
        Cols<C, NR>::load(q + (6 + a) * BC, p2);
        Cols<C, NR>::load(q + (9 + a) * BC, p3);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            C s0, s1;
            s_apply_rt(mu, p2[r], p3[r], s0, s1);
            if (!plus) { s0 = cneg(s0); s1 = cneg(s1); }
            h[0][a][r] = SMPQ_HADD(p0[r], s0);
            h[1][a][r] = SMPQ_HADD(p1[r], s1);
        }
    }
    const C *ul = U + ((size_t)mu * Vl + ls) * 9;
    const int ra = back ? 1 : 3, rb = back ? 3 : 1; // element (a, b) of W at ul[a * ra + b * rb]
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        C ur[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) ur[b] = conj_if(ul[a * ra + b * rb], back);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            C w0, w1;
#ifndef SMPQ_DF64_CHAINED
            if constexpr (std::is_same<T, df64>::value) {
                const C v0[3] = {h[0][0][r], h[0][1][r], h[0][2][r]}, v1[3] = {h[1][0][r], h[1][1][r], h[1][2][r]};
                w0 = SMPQ_HDOT(ur, v0);
                w1 = SMPQ_HDOT(ur, v1);
            } else
#endif
            {
                w0 = mkc<C>(0, 0);
                w1 = mkc<C>(0, 0);
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    w0 = cfma(ur[b], h[0][b][r], w0);
                    w1 = cfma(ur[b], h[1][b][r], w1);
                }
            }
            if (flip) {
                w0 = cneg(w0);
                w1 = cneg(w1);
            }
            acc[a][r] = SMPQ_HADD(acc[a][r], w0);
            acc[3 + a][r] = SMPQ_HADD(acc[3 + a][r], w1);
            C l0, l1;
            sdag_apply_rt(mu, w0, w1, l0, l1);
            if (!plus) { l0 = cneg(l0); l1 = cneg(l1); }
            acc[6 + a][r] = SMPQ_HADD(acc[6 + a][r], l0);
            acc[9 + a][r] = SMPQ_HADD(acc[9 + a][r], l1);
        }
    }
}

template <typename T, bool DAG, int BC, int NR = 1>
__device__ __forceinline__ void wilson_hop_rolled(const Geom &g, const typename cplx_t<T>::type *__restrict__ U,
                                                  const typename cplx_t<T>::type *__restrict__ in, int s,
                                                  typename cplx_t<T>::type acc[12][NR]) {
    typedef typename cplx_t<T>::type C;
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[c][r] = mkc<C>(0, 0);
    const SiteCoords xc(g, s);
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const int mu = k >> 1;
        const bool back = k & 1;
        const int n = g.n[mu], st = g.stride[mu], c = xc.x[mu];
        const bool edge = back ? c == 0 : c == n - 1;
        const int nb = back ? (edge ? s + (n - 1) * st : s - st) : (edge ? s - (n - 1) * st : s + st);
        const bool flip = edge && g.bcf[mu] < 0;
        // forward: (1 - g) [DAG: (1 + g)], backward: (1 + g) [DAG: (1 - g)]
        const bool plus = back != DAG;
        hop_one_rt<T, BC, NR>(mu, plus, back, U, in, g.V, nb, back ? nb : s, flip, acc);
    }
#pragma unroll
    for (int c = 0; c < 12; ++c)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[c][r] = crenorm(acc[c][r]);
}

// Float-float hop with the accumulators of the two spin rows of each half in
// packed two-lane form: upper half (acc[a], acc[3 + a]) and lower half
// (acc[6 + a], acc[9 + a]).  The colour products come out of cdot3x2_pairs in
// that form; S_mu^dag on the lower half is a lane swap (mu <= 1), a
// multiplication by i (mu = 0, 2) and a lane-1 sign (mu = 1, 2), and the
// projector sign and the boundary factor enter as sign pairs.
// MUC >= 0: the direction is that compile-time constant (the selects of S_mu
// and S_mu^dag fold away); MUC < 0: the runtime mu_rt.
// SMPQ_DF64_PACKED_PROJ=1: the projection in packed two-lane form as well.
#ifndef SMPQ_DF64_PACKED_PROJ
#define SMPQ_DF64_PACKED_PROJ 1
#endif
template <int BC, int MUC = -1>
__device__ __forceinline__ void hop_one_pairs(int mu_rt, bool plus, bool back, const df64c *__restrict__ U,
                                              const df64c *__restrict__ in, int Vl, int nb, int ls, bool flip,
                                              f2c accU[3], f2c accL[3]) {
    const int mu = MUC >= 0 ? MUC : mu_rt;
    const df64c *q = in + (size_t)nb * (12 * BC);
#if SMPQ_DF64_PACKED_PROJ
    // projection in packed form, lanes = the two spin rows: h = P + S_mu L with
    // P = (psi_0, psi_1), L = (psi_2, psi_3); S_mu is a lane swap (mu <= 1), a
    // re/im exchange (mu = 0, 2) and a pair of signs per component (times the
    // projector sign), the same exact operations as s_apply_rt and cneg
    float2 hxh[3], hxl[3], hyh[3], hyl[3];
    {
        const bool swp = mu <= 1, rot = mu == 0 || mu == 2;
        const float pm = plus ? 1.f : -1.f;
        const float2 sxp = mu == 1 ? make_float2(-pm, pm) : mu == 2 ? make_float2(pm, -pm) : make_float2(pm, pm);
        const float2 syp = mu == 0   ? make_float2(-pm, -pm)
                           : mu == 1 ? make_float2(-pm, pm)
                           : mu == 2 ? make_float2(-pm, pm)
                                     : make_float2(pm, pm);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const df64c p0 = q[a * BC], p1 = q[(3 + a) * BC], p2 = q[(6 + a) * BC], p3 = q[(9 + a) * BC];
            const df64c l0 = swp ? p3 : p2, l1 = swp ? p2 : p3;
            const df64 lx0 = rot ? l0.y : l0.x, ly0 = rot ? l0.x : l0.y, lx1 = rot ? l1.y : l1.x,
                       ly1 = rot ? l1.x : l1.y;
            const float2 lxh = __fmul2_rn(sxp, make_float2(lx0.hi, lx1.hi));
            const float2 lxl = __fmul2_rn(sxp, make_float2(lx0.lo, lx1.lo));
            const float2 lyh = __fmul2_rn(syp, make_float2(ly0.hi, ly1.hi));
            const float2 lyl = __fmul2_rn(syp, make_float2(ly0.lo, ly1.lo));
            float2 t, e;
            two_sum2(make_float2(p0.x.hi, p1.x.hi), lxh, t, e);
            hxh[a] = t;
            hxl[a] = __fadd2_rn(e, __fadd2_rn(make_float2(p0.x.lo, p1.x.lo), lxl));
            two_sum2(make_float2(p0.y.hi, p1.y.hi), lyh, t, e);
            hyh[a] = t;
            hyl[a] = __fadd2_rn(e, __fadd2_rn(make_float2(p0.y.lo, p1.y.lo), lyl));
        }
    }
#else
    df64c h0[3], h1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        df64c p0 = q[a * BC], p1 = q[(3 + a) * BC], p2 = q[(6 + a) * BC], p3 = q[(9 + a) * BC];
        df64c s0, s1;
        s_apply_rt(mu, p2, p3, s0, s1);
        if (!plus) { s0 = cneg(s0); s1 = cneg(s1); }
        h0[a] = cadd_lazy(p0, s0);
        h1[a] = cadd_lazy(p1, s1);
    }
#endif
    const df64c *ul = U + ((size_t)mu * Vl + ls) * 9;
    const int ra = back ? 1 : 3, rb = back ? 3 : 1; // element (a, b) of W at ul[a * ra + b * rb]
    const float f = flip ? -1.f : 1.f, g = plus ? f : -f, g1 = (mu == 1 || mu == 2) ? -g : g;
    const bool swp = mu <= 1, rot = mu == 0 || mu == 2;
    const float2 su = make_float2(f, f), sy = make_float2(g, g1), sx = rot ? make_float2(-g, -g1) : sy;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        df64c ur[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) ur[b] = conj_if(ul[a * ra + b * rb], back);
        float2 sr, er, si, ei;
#if SMPQ_DF64_PACKED_PROJ
        cdot3x2_packed(ur, hxh, hxl, hyh, hyl, sr, er, si, ei);
#else
        cdot3x2_pairs(ur, h0, h1, sr, er, si, ei);
#endif
        f2c_add_lazy(accU[a], su, su, sr, er, si, ei);
        if (swp) {
            sr = make_float2(sr.y, sr.x);
            er = make_float2(er.y, er.x);
            si = make_float2(si.y, si.x);
            ei = make_float2(ei.y, ei.x);
        }
        if (rot) f2c_add_lazy(accL[a], sx, sy, si, ei, sr, er);
        else f2c_add_lazy(accL[a], sx, sy, sr, er, si, ei);
    }
}

// SMPQ_DF64_MU_UNROLL=1: the 8 hops as 4 direction copies x a 2-orientation
// loop; 0: one rolled loop over all 8
#ifndef SMPQ_DF64_MU_UNROLL
#define SMPQ_DF64_MU_UNROLL 1
#endif
template <bool DAG, int BC>
__device__ __forceinline__ void wilson_hop_pairs(const Geom &g, const df64c *__restrict__ U,
                                                 const df64c *__restrict__ in, int s, df64c acc[12][1]) {
    f2c accU[3], accL[3];
    const float2 z = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 3; ++a) accU[a] = accL[a] = f2c{z, z, z, z};
    const SiteCoords xc(g, s);
#if SMPQ_DF64_MU_UNROLL
    // one copy of the hop per direction (the direction's selects fold away),
    // the two orientations in a loop: half the code of the fully unrolled hop
    auto dir = [&](auto mc) {
        constexpr int MU = decltype(mc)::value;
        const int n = g.n[MU], st = g.stride[MU], c = xc.x[MU];
#pragma unroll 1
        for (int bk = 0; bk < 2; ++bk) {
            const bool back = bk != 0;
            const bool edge = back ? c == 0 : c == n - 1;
            const int nb = back ? (edge ? s + (n - 1) * st : s - st) : (edge ? s - (n - 1) * st : s + st);
            const bool flip = edge && g.bcf[MU] < 0;
            hop_one_pairs<BC, MU>(MU, back != DAG, back, U, in, g.V, nb, back ? nb : s, flip, accU, accL);
        }
        asm volatile("" ::: "memory"); // no loads hoisted across directions (bounds the live registers)
    };
    dir(std::integral_constant<int, 0>());
    dir(std::integral_constant<int, 1>());
    dir(std::integral_constant<int, 2>());
    dir(std::integral_constant<int, 3>());
#else
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const int mu = k >> 1;
        const bool back = k & 1;
        const int n = g.n[mu], st = g.stride[mu], c = xc.x[mu];
        const bool edge = back ? c == 0 : c == n - 1;
        const int nb = back ? (edge ? s + (n - 1) * st : s - st) : (edge ? s - (n - 1) * st : s + st);
        const bool flip = edge && g.bcf[mu] < 0;
        hop_one_pairs<BC>(mu, back != DAG, back, U, in, g.V, nb, back ? nb : s, flip, accU, accL);
    }
#endif
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 xh, xl, yh, yl;
        two_sum2(accU[a].xh, accU[a].xl, xh, xl);
        two_sum2(accU[a].yh, accU[a].yl, yh, yl);
        acc[a][0] = {df64(xh.x, xl.x), df64(yh.x, yl.x)};
        acc[3 + a][0] = {df64(xh.y, xl.y), df64(yh.y, yl.y)};
        two_sum2(accL[a].xh, accL[a].xl, xh, xl);
        two_sum2(accL[a].yh, accL[a].yl, yh, yl);
        acc[6 + a][0] = {df64(xh.x, xl.x), df64(yh.x, yl.x)};
        acc[9 + a][0] = {df64(xh.y, xl.y), df64(yh.y, yl.y)};
    }
}

// Unrolled hop for FP32/FP64, rolled with packed two-lane accumulators for
// float-float (SMPQ_DF64_UNROLLED, SMPQ_DF64_UNPAIRED, SMPQ_DF64_EAGER and
// SMPQ_FP32_ROLLED switch the choice for tuning sweeps).
template <typename T, bool DAG, int BC, int NR = 1>
__device__ __forceinline__ void wilson_hop_auto(const Geom &g, const typename cplx_t<T>::type *__restrict__ U,
                                                const typename cplx_t<T>::type *__restrict__ in, int s,
                                                typename cplx_t<T>::type acc[12][NR]) {
#ifdef SMPQ_DF64_UNROLLED
    constexpr bool roll_df = false;
#else
    constexpr bool roll_df = true;
#endif
#ifdef SMPQ_FP32_ROLLED
    constexpr bool roll_f = true;
#else
    constexpr bool roll_f = false;
#endif
#if defined(SMPQ_DF64_UNPAIRED) || defined(SMPQ_DF64_EAGER)
    constexpr bool pairacc = false;
#else
    constexpr bool pairacc = true;
#endif
    if constexpr (std::is_same<T, df64>::value && roll_df && pairacc && NR == 1)
        wilson_hop_pairs<DAG, BC>(g, U, in, s, acc);
    else if constexpr ((std::is_same<T, df64>::value && roll_df) || (std::is_same<T, float>::value && roll_f))
        wilson_hop_rolled<T, DAG, BC, NR>(g, U, in, s, acc);
    else
        wilson_hop<T, DAG, BC, NR>(g, U, in, s, acc);
}

// Thread -> (tile, site, column) mapping shared by the lattice kernels:
// TPS = BC/NR threads per site and SPB sites per block;
// site = tile * SPB + tid / TPS, first column jj = (tid % TPS) * NR.
template <int BC, int NR = 1> struct TileMap {
    static constexpr int TPS = BC / NR;
    static constexpr int SPB = (256 / TPS) > 0 ? (256 / TPS) : 1;
    static constexpr int THREADS = TPS * SPB;
};
