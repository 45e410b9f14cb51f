// Wilson hopping term of D_W (Sec. 2.1, around Eq. 3) for one site and one
// right-hand side, with half-spinor projection.
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
#pragma once
#include "smpq_internal.cuh"

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

// One hop: acc += (1 + SG g_mu) W psi(nb) * f, with W = U (BACK = false) or
// U^dag (BACK = true) read from link site ls.
// `in` has component stride Vf * BC (field sites), links have site stride Vl.
template <typename T, int MU, int SG, bool BACK, int BC>
__device__ __forceinline__ void hop_one(const typename cplx_t<T>::type *__restrict__ U,
                                        const typename cplx_t<T>::type *__restrict__ in, int Vf, int Vl, int nb,
                                        int ls, T f, typename cplx_t<T>::type acc[12]) {
    typedef typename cplx_t<T>::type C;
    C p[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) p[c] = in[(size_t)(c * Vf + nb) * BC];
    // project
    C h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        C s0, s1;
        s_apply<MU>(p[6 + a], p[9 + a], s0, s1);
        if (SG > 0) { h[0][a] = cadd(p[a], s0); h[1][a] = cadd(p[3 + a], s1); }
        else { h[0][a] = csub(p[a], s0); h[1][a] = csub(p[3 + a], s1); }
    }
    // colour multiply
    C u[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) u[e] = U[(size_t)(MU * 9 + e) * Vl + ls];
    C w[2][3];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C t = mkc<C>(0, 0);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (BACK) t = cfmac(u[b * 3 + a], h[sp][b], t);
                else t = cfma(u[a * 3 + b], h[sp][b], t);
            }
            w[sp][a] = cscale(f, t);
        }
    // reconstruct
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] = cadd(acc[a], w[0][a]);
        acc[3 + a] = cadd(acc[3 + a], w[1][a]);
        C l0, l1;
        sdag_apply<MU>(w[0][a], w[1][a], l0, l1);
        if (SG > 0) { acc[6 + a] = cadd(acc[6 + a], l0); acc[9 + a] = cadd(acc[9 + a], l1); }
        else { acc[6 + a] = csub(acc[6 + a], l0); acc[9 + a] = csub(acc[9 + a], l1); }
    }
}

// SMPQ_HOP_FENCE: keep the compiler from hoisting the loads of later hops
// above earlier ones (bounds the live registers to about one neighbour).
#ifdef SMPQ_HOP_FENCE
#define SMPQ_FENCE() asm volatile("" ::: "memory")
#else
#define SMPQ_FENCE()
#endif

template <typename T, int MU, bool DAG, int BC>
__device__ __forceinline__ void hop_dir(const Geom &g, const typename cplx_t<T>::type *__restrict__ U,
                                        const typename cplx_t<T>::type *__restrict__ in, int s,
                                        typename cplx_t<T>::type acc[12]) {
    float f;
    SMPQ_FENCE();
    int nf = neighbour(g, s, MU, +1, &f);
    // forward: (1 - g) U(x) psi(x+mu)   [DAG: (1 + g)]
    hop_one<T, MU, DAG ? +1 : -1, false, BC>(U, in, g.V, g.V, nf, s, (T)f, acc);
    int nbk = neighbour(g, s, MU, -1, &f);
    SMPQ_FENCE();
    // backward: (1 + g) U(x-mu)^dag psi(x-mu)   [DAG: (1 - g)]
    hop_one<T, MU, DAG ? -1 : +1, true, BC>(U, in, g.V, g.V, nbk, nbk, (T)f, acc);
}

// acc = hop(s) for the right-hand side whose tile base pointer is `in`
// (already offset by tile and column).
template <typename T, bool DAG, int BC>
__device__ __forceinline__ void wilson_hop(const Geom &g, const typename cplx_t<T>::type *__restrict__ U,
                                           const typename cplx_t<T>::type *__restrict__ in, int s,
                                           typename cplx_t<T>::type acc[12]) {
    typedef typename cplx_t<T>::type C;
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = mkc<C>(0, 0);
    hop_dir<T, 0, DAG, BC>(g, U, in, s, acc);
    hop_dir<T, 1, DAG, BC>(g, U, in, s, acc);
    hop_dir<T, 2, DAG, BC>(g, U, in, s, acc);
    hop_dir<T, 3, DAG, BC>(g, U, in, s, acc);
}

// Thread -> (tile, site, column) mapping shared by the lattice kernels:
// blockDim.x = BC * spb threads, site = tile_site0 + threadIdx.x / BC, jj = threadIdx.x % BC.
template <int BC> struct TileMap {
    static constexpr int SPB = (256 / BC) > 0 ? (256 / BC) : 1; // sites per block
    static constexpr int THREADS = BC * SPB;
};
