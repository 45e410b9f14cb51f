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

// Shared-memory footprint of the stages (bytes), without the barriers
template <int BC, int NS> struct Dims {
    typedef TileMap<BC, 1> TM;
    static constexpr int SITE = 12 * BC;           // complex values of one site (one RHS tile)
    static constexpr int STAGE = TM::SPB * SITE;   // one stage: SPB neighbour sites
    static constexpr uint32_t SITE_BYTES = SITE * sizeof(float2);
    static constexpr size_t SMEM = (size_t)NS * STAGE * sizeof(float2) + NS * sizeof(uint64_t);
};

// Issue the copies of step k (hop k % 8 of tile tile0 + k / 8) into stage k % NS.
// Called by the 32 lanes of warp 0.
template <int BC, int NS>
__device__ __forceinline__ void issue(const Geom &g, const float2 *__restrict__ in, int tile0, int k, float2 *stages,
                                      uint64_t *bar) {
    typedef Dims<BC, NS> D;
    const int lane = threadIdx.x & 31;
    const int tile = tile0 + k / 8, h = k % 8, mu = h >> 1, st = k % NS;
    const int s0 = tile * D::TM::SPB;
    const int nvalid = min(D::TM::SPB, g.V - s0);
    if (lane == 0) {
        fence_proxy_async(); // the block's reads of this stage (before the barrier) come first
        mbar_arrive_expect_tx(&bar[st], (uint32_t)nvalid * D::SITE_BYTES);
    }
    const int n = g.n[mu], sd = g.stride[mu];
    for (int i = lane; i < nvalid; i += 32) {
        const int s = s0 + i, c = (s / sd) % n;
        const int nb = (h & 1) ? (c == 0 ? s + (n - 1) * sd : s - sd) : (c == n - 1 ? s - (n - 1) * sd : s + sd);
        bulk_g2s(stages + (size_t)st * D::STAGE + (size_t)i * D::SITE, in + (size_t)nb * D::SITE, D::SITE_BYTES,
                 &bar[st]);
    }
}

// The hop of step H (compile-time direction and orientation) for site s from
// the staged neighbour q (shared memory, this thread's column).
template <int H, bool DAG, int BC>
__device__ __forceinline__ void hop_staged(const Geom &g, const SiteCoords &xc, const float2 *__restrict__ U,
                                           const float2 *q, int s, float2 acc[12][1]) {
    constexpr int MU = H >> 1;
    constexpr bool BACK = H & 1;
    const int n = g.n[MU], sd = g.stride[MU], c = xc.x[MU];
    const bool edge = BACK ? c == 0 : c == n - 1;
    const bool flip = edge && g.bcf[MU] < 0;
    // the link of a backward hop sits on the neighbour site
    const int ls = BACK ? (edge ? s + (n - 1) * sd : s - sd) : s;
    // forward: (1 - g) U(x) psi(x+mu) [DAG: (1 + g)]; backward: (1 + g) U(x-mu)^dag psi(x-mu) [DAG: (1 - g)]
    constexpr int SG = BACK ? (DAG ? -1 : +1) : (DAG ? +1 : -1);
    hop_one<float, MU, SG, BACK, BC, 1>(U, q, g.V, g.V, 0, ls, flip, acc);
}

// Block state of a staged D_W launch: the stage buffers and barriers in
// dynamic shared memory, the block's lattice tiles, the step counter.
template <bool DAG, int BC, int NS> struct Runner {
    typedef Dims<BC, NS> D;
    float2 *stages;
    uint64_t *bar;
    const Geom &g;
    const float2 *__restrict__ U;
    const float2 *__restrict__ in; // this RHS tile of the input field (first column)
    int tile0, ntb, K;
    bool dead;
    int *err;

    __device__ Runner(unsigned char *smem, const Geom &g_, const float2 *U_, const float2 *in_, int tile0_, int ntb_,
                      int *err_)
        : g(g_), U(U_), in(in_), tile0(tile0_), ntb(ntb_), dead(false), err(err_) {
        stages = reinterpret_cast<float2 *>(smem);
        bar = reinterpret_cast<uint64_t *>(smem + (size_t)NS * D::STAGE * sizeof(float2));
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
        if (!dead && threadIdx.x < 32)
            for (int k = 0; k < NS && k < K; ++k) issue<BC, NS>(g, in, tile0, k, stages, bar);
    }

    // the 8 hops of lattice tile tl of the block for site s (valid: s < V) into acc
    __device__ __forceinline__ void hops(int tl, int s, bool valid, float2 acc[12][1]) {
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c][0] = make_float2(0.f, 0.f);
        const SiteCoords xc(g, valid ? s : 0);
        const int i = threadIdx.x / BC, jj = threadIdx.x % BC;
        auto step = [&](auto hc) {
            constexpr int H = decltype(hc)::value;
            const int k = tl * 8 + H, st = k % NS;
            bool ok = true;
            if (!dead) ok = mbar_wait(&bar[st], (uint32_t)((k / NS) & 1), WAIT_LIMIT);
            if (!dead && valid)
                hop_staged<H, DAG, BC>(g, xc, U, stages + (size_t)st * D::STAGE + (size_t)i * D::SITE + jj, s, acc);
            if (__syncthreads_or(!ok)) {
                if (!dead) fail(k);
                return;
            }
            if (!dead && threadIdx.x < 32 && k + NS < K) issue<BC, NS>(g, in, tile0, k + NS, stages, bar);
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
        __syncthreads();
    }
};

} // namespace stage
