// FP32 Wilson hopping term with the neighbour sites staged in shared memory
// by bulk asynchronous copies (the TMA engine, cp.async.bulk), completed on
// mbarriers.  The arithmetic is that of hop_one (wilson.cuh, Sec. 2.1, Eq. 3);
// only where the neighbour spinors come from changes.
//
// Why: the one-thread-per-site-and-column FP32 D_W is latency bound (ncu: the
// leading stall is the L1TEX scoreboard, 37 % occupancy limited by registers,
// DRAM at about half its peak).  Here a block's neighbour data for the next
// hops is in flight in the copy engine while the threads compute the current
// hop, so the bytes in flight no longer depend on registers.
//
// Layout: a field tile stores a site as 12 * BC contiguous complex values
// ([component][column]), so the neighbour of a site in one direction is one
// contiguous copy of 96 * BC bytes (a multiple of 16, as cp.async.bulk needs;
// every field and tile offset is a multiple of 16 bytes as well).  A block
// handles SPB consecutive sites x BC columns per lattice tile; step k of the
// block is hop (k mod 8) of its (k / 8)-th lattice tile, and its SPB
// neighbour sites go to stage buffer k mod NS.  Warp 0 issues the copies of
// step k + NS once every thread has finished step k (one block barrier per
// hop), so NS - 1 steps of copies are in flight during each hop.
//
// Every wait is bounded (about a second of SM clock); a wait that runs out
// marks the launch as failed (atomicOr on *err), the block stops computing
// (its results are then meaningless, and the host reports the error), waits
// again with a bound for the copies it still has in flight, and runs to its
// end so that the fused scalar steps keep their arrival protocol.  A block
// that starts after *err is set copies and waits for nothing.
#pragma once
#include <stdint.h>

#include "device.cuh"
#include "wilson.cuh"

namespace stage {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the copy engine
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// the generic-proxy accesses of this thread before the async-proxy copies after
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// arrive on the barrier and add `bytes` to the transaction count of its phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing `bytes` transactions on bar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// wait for the phase with the given parity to complete, for at most `limit`
// SM clock cycles; false if it did not
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > limit) return false;
    }
}

constexpr int NSTAGE = 3; // stage buffers: two steps of copies in flight during each hop
constexpr long long WAIT_LIMIT = 1LL << 31;   // about a second at 2 GHz
constexpr long long CLEANUP_LIMIT = 1LL << 28; // per outstanding stage after a failure

// 8-byte asynchronous copy global -> shared (the FP32 links: 72 bytes each, so
// not aligned for the bulk engine), completed per thread by commit / wait groups
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ float2 lds2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}


// Shared-memory layout of the stages: NS field stages of SPB sites, NS link
// stages of SPB links (9 complex values each), NS barriers
template <int BC, int NS> struct Dims {
    typedef TileMap<BC, 1> TM;
    static constexpr int SITE = 12 * BC;           // complex values of one site (one RHS tile)
    static constexpr int STAGE = TM::SPB * SITE;   // one field stage: SPB neighbour sites
    static constexpr int LSTAGE = TM::SPB * 9;     // one link stage: the link of each site's hop
    static constexpr uint32_t SITE_BYTES = SITE * sizeof(float2);
    static constexpr size_t LINK_OFF = (size_t)NS * STAGE * sizeof(float2);
    static constexpr size_t BAR_OFF = LINK_OFF + (size_t)NS * LSTAGE * sizeof(float2);
    static constexpr size_t SMEM = BAR_OFF + NS * sizeof(uint64_t);
};

// Issue the copies of step k (hop k % 8 of tile tile0 + k / 8) into stage
// k % NS: lane i < SPB copies the neighbour site of block site i (bulk copy on
// the stage's barrier) and the hop's link (nine 8-byte copies); every lane
// then commits one copy group, so that group j of a lane is always step j.
// Called by the 32 lanes of warp 0, with k < K.
template <int BC, int NS>
__device__ __forceinline__ void issue(const Geom &g, const float2 *__restrict__ U, const float2 *__restrict__ in,
                                      int tile0, int k, unsigned char *smem, uint64_t *bar) {
    typedef Dims<BC, NS> D;
    const int lane = threadIdx.x & 31;
    const int tile = tile0 + k / 8, h = k % 8, mu = h >> 1, st = k % NS;
    const bool back = h & 1;
    const int s0 = tile * D::TM::SPB;
    const int nvalid = min(D::TM::SPB, g.V - s0);
    if (lane == 0) {
        fence_proxy_async(); // the block's reads of this stage (before the barrier) come first
        mbar_arrive_expect_tx(&bar[st], (uint32_t)nvalid * D::SITE_BYTES);
    }
    const int n = g.n[mu], sd = g.stride[mu];
    for (int i = lane; i < nvalid; i += 32) {
        const int s = s0 + i, c = (s / sd) % n;
        const int nb = back ? (c == 0 ? s + (n - 1) * sd : s - sd) : (c == n - 1 ? s - (n - 1) * sd : s + sd);
        bulk_g2s(smem + ((size_t)st * D::STAGE + (size_t)i * D::SITE) * sizeof(float2), in + (size_t)nb * D::SITE,
                 D::SITE_BYTES, &bar[st]);
        // the link of a forward hop sits on the site, of a backward hop on the neighbour
        const float2 *u = U + ((size_t)mu * g.V + (back ? nb : s)) * 9;
        const uint32_t dst = smem_u32(smem + D::LINK_OFF + ((size_t)st * D::LSTAGE + (size_t)i * 9) * sizeof(float2));
#pragma unroll
        for (int e = 0; e < 9; ++e) cp_async8(dst + e * sizeof(float2), u + e);
    }
    cp_async_commit();
}

// One hop for one column, neighbour spinor and link read from the stages
// (shared addresses q: component 0 of this column, components BC apart; ul:
// the 9 link elements).  The arithmetic and its order are those of hop_one.
template <int MU, int SG, bool BACK, int BC>
__device__ __forceinline__ void hop_smem(uint32_t q, uint32_t ul, bool flip, float2 acc[12][1]) {
    constexpr uint32_t CS = BC * sizeof(float2); // bytes between components
    float2 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float2 p0 = lds2(q + a * CS), p1 = lds2(q + (3 + a) * CS);
        const float2 p2 = lds2(q + (6 + a) * CS), p3 = lds2(q + (9 + a) * CS);
        float2 s0, s1;
        s_apply<MU>(p2, p3, s0, s1);
        if (SG > 0) { h[0][a] = cadd(p0, s0); h[1][a] = cadd(p1, s1); }
        else { h[0][a] = csub(p0, s0); h[1][a] = csub(p1, s1); }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 ur[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) ur[b] = lds2(ul + (BACK ? b * 3 + a : a * 3 + b) * sizeof(float2));
        float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (BACK) {
                w0 = cfmac(ur[b], h[0][b], w0);
                w1 = cfmac(ur[b], h[1][b], w1);
            } else {
                w0 = cfma(ur[b], h[0][b], w0);
                w1 = cfma(ur[b], h[1][b], w1);
            }
        }
        if (flip) {
            w0 = cneg(w0);
            w1 = cneg(w1);
        }
        acc[a][0] = cadd(acc[a][0], w0);
        acc[3 + a][0] = cadd(acc[3 + a][0], w1);
        float2 l0, l1;
        sdag_apply<MU>(w0, w1, l0, l1);
        if (SG > 0) { acc[6 + a][0] = cadd(acc[6 + a][0], l0); acc[9 + a][0] = cadd(acc[9 + a][0], l1); }
        else { acc[6 + a][0] = csub(acc[6 + a][0], l0); acc[9 + a][0] = csub(acc[9 + a][0], l1); }
    }
}

// Block state of a staged D_W launch: the stage buffers and barriers in
// dynamic shared memory, the block's lattice tiles, the step counter.
template <bool DAG, int BC, int NS> struct Runner {
    typedef Dims<BC, NS> D;
    unsigned char *smem;
    uint64_t *bar;
    const Geom &g;
    const float2 *__restrict__ U;
    const float2 *__restrict__ in; // this RHS tile of the input field (first column)
    int tile0, ntb, K;
    bool dead;
    int *err;

    __device__ Runner(unsigned char *smem_, const Geom &g_, const float2 *U_, const float2 *in_, int tile0_, int ntb_,
                      int *err_)
        : smem(smem_), g(g_), U(U_), in(in_), tile0(tile0_), ntb(ntb_), dead(false), err(err_) {
        bar = reinterpret_cast<uint64_t *>(smem + D::BAR_OFF);
        K = 8 * max(ntb, 0);
        bool failed = false;
        if (threadIdx.x == 0) {
            for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
            fence_barrier_init();
            failed = *(volatile int *)err != 0;
        }
        // once any block of the launch (or an earlier one) has timed out, the
        // block issues and waits for nothing: a failure costs one round of blocks
        dead = __syncthreads_or(failed) != 0;
        if (!dead && threadIdx.x < 32) {
            for (int k = 0; k < NS; ++k) {
                if (k < K) issue<BC, NS>(g, U, in, tile0, k, smem, bar);
                else cp_async_commit();
            }
            cp_async_wait<NS - 1>(); // the links of step 0
        }
        __syncthreads();
    }

    // the 8 hops of lattice tile tl of the block for site s (valid: s < V) into acc
    __device__ __forceinline__ void hops(int tl, int s, bool valid, float2 acc[12][1]) {
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c][0] = make_float2(0.f, 0.f);
        // boundary signs of the 8 hops of this site (antiperiodic directions)
        unsigned flips = 0;
        {
            const SiteCoords xc(g, valid ? s : 0);
#pragma unroll
            for (int mu = 0; mu < 4; ++mu)
                if (g.bcf[mu] < 0) {
                    if (xc.x[mu] == g.n[mu] - 1) flips |= 1u << (2 * mu);
                    if (xc.x[mu] == 0) flips |= 1u << (2 * mu + 1);
                }
        }
        const int i = threadIdx.x / BC, jj = threadIdx.x % BC;
        const uint32_t q0 = smem_u32(smem) + (uint32_t)((i * D::SITE + jj) * sizeof(float2));
        const uint32_t u0 = smem_u32(smem + D::LINK_OFF) + (uint32_t)(i * 9 * sizeof(float2));
        auto step = [&](auto hc) {
            constexpr int H = decltype(hc)::value;
            constexpr int MU = H >> 1;
            constexpr bool BACK = H & 1;
            // forward: (1 - g) U(x) psi(x+mu) [DAG: (1 + g)]; backward: (1 + g) U(x-mu)^dag psi(x-mu) [DAG: (1 - g)]
            constexpr int SG = BACK ? (DAG ? -1 : +1) : (DAG ? +1 : -1);
            const int k = tl * 8 + H, st = k % NS;
            bool ok = true;
            if (!dead) ok = mbar_wait(&bar[st], (uint32_t)((k / NS) & 1), WAIT_LIMIT);
            if (!dead && valid)
                hop_smem<MU, SG, BACK, BC>(q0 + (uint32_t)(st * D::STAGE * sizeof(float2)),
                                           u0 + (uint32_t)(st * D::LSTAGE * sizeof(float2)), (flips >> H) & 1u, acc);
            // warp 0: the links of step k + 1 have arrived (its group; the
            // later NS - 2 may still be in flight) before the barrier
            if (!dead && threadIdx.x < 32) cp_async_wait<NS - 2>();
            if (__syncthreads_or(!ok)) {
                if (!dead) fail(k);
                return;
            }
            if (!dead && threadIdx.x < 32) {
                if (k + NS < K) issue<BC, NS>(g, U, in, tile0, k + NS, smem, bar);
                else cp_async_commit(); // an empty group keeps group j = step j
            }
        };
        step(std::integral_constant<int, 0>());
        step(std::integral_constant<int, 1>());
        step(std::integral_constant<int, 2>());
        step(std::integral_constant<int, 3>());
        step(std::integral_constant<int, 4>());
        step(std::integral_constant<int, 5>());
        step(std::integral_constant<int, 6>());
        step(std::integral_constant<int, 7>());
    }

    // a wait ran out at step k (block-uniform): report it, wait with a bound
    // for the copies still in flight (steps k .. k + NS - 1), stop computing
    __device__ void fail(int k) {
        dead = true;
        if (threadIdx.x == 0) {
            atomicOr(err, 1);
            for (int kk = k; kk < k + NS && kk < K; ++kk)
                mbar_wait(&bar[kk % NS], (uint32_t)((kk / NS) & 1), CLEANUP_LIMIT);
        }
        if (threadIdx.x < 32) cp_async_wait<0>();
        __syncthreads();
    }
};

// ------------------------------------------------------------------ float-float
// The float-float D_W (16-byte complex values) staged the same way, with two
// stages (one step of copies in flight: a float-float hop is long enough to
// cover it, and two 46 KB stages leave room for two blocks per SM).  The link
// of a hop (9 x 16 bytes) is 16-byte aligned, so it travels by bulk copy on
// the same barrier as the neighbour site.  The hop loop stays rolled (the
// unrolled float-float hop overflows the instruction cache) and uses the
// packed two-lane hop of wilson.cuh with shared-memory operands.
template <int BC, int NS> struct DimsDF {
    typedef TileMap<BC, 1> TM;
    static constexpr int SITE = 12 * BC;
    static constexpr int STAGE = TM::SPB * SITE;
    static constexpr int LSTAGE = TM::SPB * 9;
    static constexpr uint32_t SITE_BYTES = SITE * sizeof(df64c);
    static constexpr uint32_t LINK_BYTES = 9 * sizeof(df64c);
    static constexpr size_t LINK_OFF = (size_t)NS * STAGE * sizeof(df64c);
    static constexpr size_t BAR_OFF = LINK_OFF + (size_t)NS * LSTAGE * sizeof(df64c);
    static constexpr size_t SMEM = BAR_OFF + NS * sizeof(uint64_t);
};
constexpr int NSTAGE_DF = 2;

template <int BC, int NS>
__device__ __forceinline__ void issue_df(const Geom &g, const df64c *__restrict__ U, const df64c *__restrict__ in,
                                         int tile0, int k, unsigned char *smem, uint64_t *bar) {
    typedef DimsDF<BC, NS> D;
    const int lane = threadIdx.x & 31;
    const int tile = tile0 + k / 8, h = k % 8, mu = h >> 1, st = k % NS;
    const bool back = h & 1;
    const int s0 = tile * D::TM::SPB;
    const int nvalid = min(D::TM::SPB, g.V - s0);
    if (lane == 0) {
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[st], (uint32_t)nvalid * (D::SITE_BYTES + D::LINK_BYTES));
    }
    const int n = g.n[mu], sd = g.stride[mu];
    for (int i = lane; i < nvalid; i += 32) {
        const int s = s0 + i, c = (s / sd) % n;
        const int nb = back ? (c == 0 ? s + (n - 1) * sd : s - sd) : (c == n - 1 ? s - (n - 1) * sd : s + sd);
        bulk_g2s(smem + ((size_t)st * D::STAGE + (size_t)i * D::SITE) * sizeof(df64c), in + (size_t)nb * D::SITE,
                 D::SITE_BYTES, &bar[st]);
        bulk_g2s(smem + D::LINK_OFF + ((size_t)st * D::LSTAGE + (size_t)i * 9) * sizeof(df64c),
                 U + ((size_t)mu * g.V + (back ? nb : s)) * 9, D::LINK_BYTES, &bar[st]);
    }
}

template <bool DAG, int BC, int NS> struct RunnerDF {
    typedef DimsDF<BC, NS> D;
    unsigned char *smem;
    uint64_t *bar;
    const Geom &g;
    const df64c *__restrict__ U;
    const df64c *__restrict__ in;
    int tile0, ntb, K;
    bool dead;
    int *err;

    __device__ RunnerDF(unsigned char *smem_, const Geom &g_, const df64c *U_, const df64c *in_, int tile0_,
                        int ntb_, int *err_)
        : smem(smem_), g(g_), U(U_), in(in_), tile0(tile0_), ntb(ntb_), dead(false), err(err_) {
        bar = reinterpret_cast<uint64_t *>(smem + D::BAR_OFF);
        K = 8 * max(ntb, 0);
        bool failed = false;
        if (threadIdx.x == 0) {
            for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
            fence_barrier_init();
            failed = *(volatile int *)err != 0;
        }
        dead = __syncthreads_or(failed) != 0;
        if (!dead && threadIdx.x < 32)
            for (int k = 0; k < NS && k < K; ++k) issue_df<BC, NS>(g, U, in, tile0, k, smem, bar);
    }

    // the 8 hops of lattice tile tl for site s (valid: s < V): acc = hop(s)
    __device__ __forceinline__ void hops(int tl, int s, bool valid, df64c acc[12][1]) {
        f2c accU[3], accL[3];
        const float2 z = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < 3; ++a) accU[a] = accL[a] = f2c{z, z, z, z};
        const SiteCoords xc(g, valid ? s : 0);
        const int i = threadIdx.x / BC, jj = threadIdx.x % BC;
        const df64c *qs = reinterpret_cast<const df64c *>(smem) + (size_t)i * D::SITE + jj;
        const df64c *us = reinterpret_cast<const df64c *>(smem + D::LINK_OFF) + (size_t)i * 9;
#pragma unroll 1
        for (int h = 0; h < 8; ++h) {
            const int k = tl * 8 + h, st = k % NS;
            bool ok = true;
            if (!dead) ok = mbar_wait(&bar[st], (uint32_t)((k / NS) & 1), WAIT_LIMIT);
            if (!dead && valid) {
                const int mu = h >> 1;
                const bool back = h & 1;
                const bool edge = back ? xc.x[mu] == 0 : xc.x[mu] == g.n[mu] - 1;
                const bool flip = edge && g.bcf[mu] < 0;
                // forward: (1 - g) [DAG: (1 + g)], backward: (1 + g) [DAG: (1 - g)]
                hop_one_pairs<BC>(mu, back != DAG, back, us + (size_t)st * D::LSTAGE, qs + (size_t)st * D::STAGE, 0,
                                  0, 0, flip, accU, accL);
            }
            if (__syncthreads_or(!ok)) {
                if (!dead) fail(k);
                continue;
            }
            if (!dead && threadIdx.x < 32 && k + NS < K) issue_df<BC, NS>(g, U, in, tile0, k + NS, smem, bar);
        }
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

    __device__ void fail(int k) {
        dead = true;
        if (threadIdx.x == 0) {
            atomicOr(err, 1);
            for (int kk = k; kk < k + NS && kk < K; ++kk)
                mbar_wait(&bar[kk % NS], (uint32_t)((kk / NS) & 1), CLEANUP_LIMIT);
        }
        __syncthreads();
    }
};

} // namespace stage
