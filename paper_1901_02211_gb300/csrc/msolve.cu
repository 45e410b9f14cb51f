// Multi-shift CG for (D_W^dag D_W + q_i) x_i = b, all shifts in one Krylov
// space (Sec. 2.1, Eqs. 6-8; Frommer et al. 1995, Jegerlehner hep-lat/9612014),
// for a batch of B right-hand sides, accumulating y = sum_i c_i x_i (Eq. 4) on
// the support the trace needs.
//
// One iteration is three launches, with no host synchronisation:
//   A   t = D_W p, per-block partials |t|^2, |p|^2; the last block to finish
//       an RHS tile sums the tile's partials and runs the first scalar step of
//       its columns: alpha = <r,r> / (|t|^2 + s0 |p|^2), zeta_{k+1} and
//       alpha_i of every shift
//   B   r -= alpha (D_W^dag t + s0 p) [x_lo += alpha p], partials |r|^2; the
//       last block of a tile runs the second scalar step: beta, beta_i,
//       convergence |zeta_i| ||r|| <= tol ||b||, residual-replacement request
//   YP  on the support: y += c_i alpha_i p_i, p_i = zeta_{k+1} r + beta_i p_i;
//       on the lattice: p = r + beta p [x += alpha p for the true residual]
// The "last block" is found with one atomic counter per RHS tile (the CUDA
// threadfence-reduction pattern): no block ever waits for another.
// Base vectors (p, t, r) live on the whole lattice in the iteration precision T.
// Shifted directions p_i are pointwise in x (the matrix never touches them),
// so they are kept only where y is read later: the 9-site star around every
// site of the right-hand side's colour class (full lattice for smpq_apply_dov).
// FP32 path: x_hi (FP64) += x_lo at every residual replacement, where the FP64
// residual b - (A + s0) x_hi replaces r (reliable updates, Sleijpen & van der
// Vorst 1996); scalars, reductions and y stay FP64 throughout.
//
// Reductions are deterministic: per-block partial sums in a fixed tree/sequence,
// then a fixed-order sum over the blocks of a tile in the tile's last block.
#include <algorithm>
#include <cstdio>
#include <cmath>

#include "half.cuh"
#include "smpq_internal.cuh"
#include "stage.cuh"
#include "wilson.cuh"

namespace {

// Each block of a lattice kernel handles TPB consecutive tiles of one RHS
// tile, and blocks are numbered site-major inside an RHS tile, so the blocks
// resident at any moment cover a narrow band of the lattice for few RHS tiles:
// the +-t neighbours (V/n_t sites away) are still in L2 when they are read.
// (The D_W kernels take the count as an argument, chosen by the autotuner.)
constexpr int TPB = 4;

// minimum resident blocks per SM requested from the register allocator for
// the FP32 lattice kernels (240-thread blocks: 2 -> <= 136 registers, 3 -> <= 91)
#ifndef SMPQ_FP32_MIN_BLOCKS
#define SMPQ_FP32_MIN_BLOCKS 3
#endif
template <typename T> struct MinBlocks { static constexpr int value = SMPQ_FP32_MIN_BLOCKS; };
template <> struct MinBlocks<double> { static constexpr int value = 1; };
#ifndef SMPQ_DF64_MIN_BLOCKS
#define SMPQ_DF64_MIN_BLOCKS 2
#endif
template <> struct MinBlocks<df64> { static constexpr int value = SMPQ_DF64_MIN_BLOCKS; };

// link copy matching the iteration precision
template <typename T> struct Links;
template <> struct Links<double> { static const void *get(const smpq_ctx *c) { return c->U64.p; } };
template <> struct Links<float> { static const void *get(const smpq_ctx *c) { return c->U32.p; } };
template <> struct Links<df64> { static const void *get(const smpq_ctx *c) { return c->Udf.p; } };


// ------------------------------------------------------------------ block reduction per column
template <int BC>
__device__ __forceinline__ double block_sum(double v, double *sm) {
    constexpr int THREADS = TileMap<BC>::THREADS;
    double s = 0;
    if constexpr (32 % BC == 0) {
#pragma unroll
        for (int o = 16; o >= BC; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane < BC) sm[warp * BC + lane] = v;
        __syncthreads();
        if (threadIdx.x < BC)
            for (int w = 0; w < THREADS / 32; ++w) s += sm[w * BC + threadIdx.x];
        __syncthreads();
    } else {
        sm[threadIdx.x] = v;
        __syncthreads();
        if (threadIdx.x < BC)
            for (int k = threadIdx.x; k < THREADS; k += BC) s += sm[k];
        __syncthreads();
    }
    return s;
}

constexpr int NFLAGS = 5; // the flags the host reads after each check interval
struct Scal {
    double *rr, *bb, *alpha, *beta, *alpha_prev, *beta_prev, *rr_ref; // [B]
    int *act_rhs, *upd_rhs, *iters;                                  // [B]
    double *zeta, *zeta_prev, *zeta_new, *alpha_s, *beta_s;          // [n][B]
    int *act, *upd;                                                  // [n][B]
    int *flags; // [0] active rhs count, [1] residual replacement requested, [2] breakdown,
                // [3] active rhs still above the precision-switch residual,
                // [4] a staging wait of the FP32 D_W ran out (stage.cuh)
    double *hist; // Lanczos: [2][hist_len] alpha_k, beta_k of rhs 0 (nullable)
    int hist_len;
    int *iter_counter; // [1] global iteration count (for the history index)
};

// source value of component c of rhs j at site s
struct Source {
    const int *colour;     // [V] (class-based sources)
    const int *src_class;  // [B] colour class carrying rhs j (-1: zero source)
    const int *src_comp;   // [B] spin*3 + colour index of rhs j
    const double2 *b64;    // tiled FP64 explicit source (nullable)
};

template <int BC>
__device__ __forceinline__ double2 source_at(const Source &src, int V, int s, int c, int j, size_t tiled_idx) {
    if (src.b64) return src.b64[tiled_idx];
    int cl = src.src_class[j];
    return make_double2((cl >= 0 && src.colour[s] == cl && c == src.src_comp[j]) ? 1.0 : 0.0, 0.0);
}

// ------------------------------------------------------------------ the lattices of a launch
// The RHS tiles of a launch (blockIdx.y) belong to one lattice, or to several
// of different sizes (the uneven batch of smpq_compute_qx_batch): lattice l
// owns the tiles from chunk0_l on, and its part of every field buffer starts
// at element f0_l.  The iteration kernels take this table; M = false is the
// one-lattice form (entry 0, known at compile time).
constexpr int MAX_LAT = 4;
struct Lat {
    Geom g;
    const void *U;  // links in the launch's precision
    long long f0;   // first element (complex value) of the lattice's fields
    long long p0;   // first partial-sum row of the lattice in this launch
    int chunk0;     // first RHS tile
    int G;          // blocks per tile in this launch (launch YP: lattice blocks)
    double s0;      // base (smallest) shift of the lattice's rational
    int n_sup, Gs;  // launch YP: support entries per rhs, support blocks per tile
    int B;          // right-hand sides of the lattice
    const int *supsite;
    long long sup0; // first element of the lattice's support fields (y; ps shift by shift)
};
struct Lats {
    int n;
    Lat l[MAX_LAT];
};
template <bool M> __device__ __forceinline__ int lat_index(const Lats &L) {
    if constexpr (!M) return 0;
    int l = 0;
    while (l + 1 < L.n && (int)blockIdx.y >= L.l[l + 1].chunk0) ++l;
    return l;
}

// ------------------------------------------------------------------ scalar steps (one thread per column)
// First scalar step of column j: alpha and the shift recurrences zeta_{k+1},
// alpha_i (tt = |D_W p|^2, pp = |p|^2, so <p, A p> = tt + s0 pp).
__device__ void s1_column(int j, double tt, double pp, const Scal &sc, const ShiftParams &sp, int B) {
    if (j == 0) {
        sc.flags[0] = 0;
        sc.flags[3] = 0;
        if (sc.hist) {
            int it = sc.iter_counter[0];
            if (it < sc.hist_len) sc.hist[it] = 0; // filled below when rhs 0 is active
        }
    }
    if (!sc.act_rhs[j]) {
        sc.alpha[j] = 0;
        sc.upd_rhs[j] = 0;
        for (int i = 0; i < sp.n; ++i) { sc.upd[i * B + j] = 0; sc.alpha_s[i * B + j] = 0; }
        return;
    }
    double pAp = tt + sp.s0 * pp;
    if (!(pAp > 0) || !isfinite(pAp)) {
        atomicOr(&sc.flags[2], 1);
        sc.alpha[j] = 0;
        sc.upd_rhs[j] = 0;
        sc.act_rhs[j] = 0;
        for (int i = 0; i < sp.n; ++i) { sc.upd[i * B + j] = 0; sc.alpha_s[i * B + j] = 0; }
        return;
    }
    double a = sc.rr[j] / pAp;
    sc.alpha[j] = a;
    sc.upd_rhs[j] = 1;
    if (sc.hist && j == 0) {
        int it = sc.iter_counter[0];
        if (it < sc.hist_len) sc.hist[it] = a;
    }
    double ap = sc.alpha_prev[j], bp = sc.beta_prev[j];
    for (int i = 0; i < sp.n; ++i) {
        int ix = i * B + j;
        if (!sc.act[ix]) { sc.upd[ix] = 0; sc.alpha_s[ix] = 0; continue; }
        double z = sc.zeta[ix], zp = sc.zeta_prev[ix];
        double den = a * bp * (zp - z) + zp * ap * (1.0 + sp.sig[i] * a);
        double zn = z * zp * ap / den;
        sc.zeta_new[ix] = zn;
        sc.alpha_s[ix] = a * zn / z;
        sc.upd[ix] = 1;
    }
}

// Second scalar step of column j (rrn = |r_{k+1}|^2): beta, beta_i, the
// convergence of every shift, the residual-replacement request and the count
// of columns still above the precision-switch residual.
__device__ void s2_column(int j, double rrn, const Scal &sc, const ShiftParams &sp, int B, double tol2,
                          double delta2, double theta2) {
    if (j == 0) {
        if (sc.hist) {
            int it = sc.iter_counter[0];
            if (it < sc.hist_len) sc.hist[sc.hist_len + it] = sc.upd_rhs[0] ? rrn / sc.rr[0] : 0.0;
        }
        sc.iter_counter[0] += 1;
    }
    if (!sc.upd_rhs[j]) return;
    double b = rrn / sc.rr[j];
    sc.beta[j] = b;
    int any = 0;
    double bb = sc.bb[j];
    for (int i = 0; i < sp.n; ++i) {
        int ix = i * B + j;
        if (!sc.upd[ix]) { any |= sc.act[ix]; continue; }
        double z = sc.zeta[ix], zn = sc.zeta_new[ix];
        double q = zn / z;
        sc.beta_s[ix] = b * q * q;
        sc.zeta_prev[ix] = z;
        sc.zeta[ix] = zn;
        int a = zn * zn * rrn > tol2 * bb;
        sc.act[ix] = a;
        any |= a;
    }
    sc.alpha_prev[j] = sc.alpha[j];
    sc.beta_prev[j] = b;
    sc.rr[j] = rrn;
    sc.iters[j] += 1;
    sc.act_rhs[j] = any;
    if (any) atomicAdd(&sc.flags[0], 1);
    if (delta2 > 0 && rrn < delta2 * sc.rr_ref[j]) atomicOr(&sc.flags[1], 1);
    if (any && rrn > theta2 * bb) atomicAdd(&sc.flags[3], 1); // still above the precision switch
}

// What the lattice kernels A and B need for the scalar step of an RHS tile.
// count == nullptr: no scalar step (the autotuner's timing launches).
struct Fuse {
    int *count; // [tiles] blocks of the tile that have stored their partials; back to 0 after each launch
    Scal sc;
    const ShiftParams *sp; // [lattices] each lattice's shifts (device memory)
    int B;                 // right-hand sides of the solve (stride of the shift-major scalars)
    double tol2, delta2, theta2; // (second step only)
};

// Called by every thread of a block after its partial sums are stored: true
// in every thread of the block that arrives last among the G blocks of RHS
// tile blockIdx.y.  The threads that stored partials (wrote) fence them before
// the arrival count, so the last block sees every partial of its tile; the
// other threads' stores need no fence (the next launch sees them).
__device__ __forceinline__ bool last_block_of_tile(int *count, int G, bool wrote) {
    __shared__ int last;
    if (wrote) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int ticket = atomicAdd(&count[blockIdx.y], 1);
        last = ticket == G - 1;
        if (last) count[blockIdx.y] = 0; // every block of the tile has arrived: reset for the next launch
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Sum over the G blocks of an RHS tile (partial rows prow...) of each column, in
// a fixed order (NT / BC lanes per column, then the lanes in order); every
// thread of the block calls it, threads < BC receive their column's total.
template <int BC, int NT> __device__ double tile_sum(const double *part, size_t prow, int G, double *sm) {
    constexpr int K = NT / BC;
    const int t = threadIdx.x, jj = t % BC, k = t / BC;
    double v = 0;
    if (k < K)
        for (int b = k; b < G; b += K) v += __ldcg(part + (prow + b) * BC + jj);
    if (k < K) sm[t] = v;
    __syncthreads();
    double tot = 0;
    if (t < BC)
        for (int q = 0; q < K; ++q) tot += sm[q * BC + t];
    __syncthreads();
    return tot;
}

// end of lattice kernel A: the tile's last block runs the first scalar step
// (lattice l, its tile's partial rows from prow)
template <int BC, int NT>
__device__ __forceinline__ void fuse_step1(const Fuse &f, int l, const double *part_t, const double *part_p,
                                           size_t prow, int G, double *sm) {
    if (!f.count || !last_block_of_tile(f.count, G, threadIdx.x < BC)) return;
    const double tt = tile_sum<BC, NT>(part_t, prow, G, sm);
    const double pp = tile_sum<BC, NT>(part_p, prow, G, sm);
    if (threadIdx.x < BC) s1_column(blockIdx.y * BC + threadIdx.x, tt, pp, f.sc, f.sp[l], f.B);
}
// end of lattice kernel B: the tile's last block runs the second scalar step
template <int BC, int NT>
__device__ __forceinline__ void fuse_step2(const Fuse &f, int l, const double *part_r, size_t prow, int G,
                                           double *sm) {
    if (!f.count || !last_block_of_tile(f.count, G, threadIdx.x < BC)) return;
    const double rr = tile_sum<BC, NT>(part_r, prow, G, sm);
    if (threadIdx.x < BC)
        s2_column(blockIdx.y * BC + threadIdx.x, rr, f.sc, f.sp[l], f.B, f.tol2, f.delta2, f.theta2);
}

// ------------------------------------------------------------------ lattice kernels
template <typename T, int BC>
__global__ void __launch_bounds__(TileMap<BC>::THREADS)
    k_init(Geom g, Source src, typename cplx_t<T>::type *r, typename cplx_t<T>::type *p,
           typename cplx_t<T>::type *xlo, df64c *xhi, double *part, int G) {
    typedef typename cplx_t<T>::type C;
    __shared__ double sm[TileMap<BC>::THREADS];
    const int jj = threadIdx.x % BC, chunk = blockIdx.y, j = chunk * BC + jj;
    const size_t base = (size_t)chunk * 12 * g.V * BC + jj;
    const int ntiles = (g.V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    double acc = 0;
    for (int tile = blockIdx.x * TPB, tend = min(ntiles, tile + TPB); tile < tend; ++tile) {
        int s = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (s >= g.V) continue;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            size_t o = base + ((size_t)s * 12 + c) * BC;
            double2 b = source_at<BC>(src, g.V, s, c, j, o);
            C v = mkc<C>(b.x, b.y);
            r[o] = v;
            p[o] = v;
            if (xlo) xlo[o] = mkc<C>(0, 0);
            if (xhi) xhi[o] = df64c{df64(0.f), df64(0.f)};
            acc += b.x * b.x + b.y * b.y;
        }
    }
    double s = block_sum<BC>(acc, sm);
    if (threadIdx.x < BC) part[((size_t)chunk * G + blockIdx.x) * BC + threadIdx.x] = s;
}

// per-column sums over a block of the NR-column kernels (sites x columns in
// shared memory, then a fixed-order sum down each column); threads < BC return
// the total of column threadIdx.x
template <int BC, int NR>
__device__ __forceinline__ double block_sum_cols(const double v[NR], double *sm) {
    constexpr int TPS = TileMap<BC, NR>::TPS, SPB = TileMap<BC, NR>::SPB;
    const int row = threadIdx.x / TPS, col0 = (threadIdx.x % TPS) * NR;
#pragma unroll
    for (int r = 0; r < NR; ++r) sm[row * BC + col0 + r] = v[r];
    __syncthreads();
    double s = 0;
    if (threadIdx.x < BC)
        for (int k = 0; k < SPB; ++k) s += sm[k * BC + threadIdx.x];
    __syncthreads();
    return s;
}

template <int BC, int NR>
__device__ __forceinline__ double block_total(const double v[NR], double *sm) {
    if constexpr (NR == 1) return block_sum<BC>(v[0], sm);
    else return block_sum_cols<BC, NR>(v, sm);
}

template <int BC, int NR> struct SmemCols {
    static constexpr int N = TileMap<BC, NR>::THREADS > TileMap<BC, NR>::SPB * BC ? TileMap<BC, NR>::THREADS
                                                                                   : TileMap<BC, NR>::SPB * BC;
};

// t = D_W p ; partials |t|^2 -> part_t, |p|^2 -> part_p (NR columns per thread)
template <typename T, int BC, int NR, bool M>
__global__ void __launch_bounds__(TileMap<BC, NR>::THREADS, MinBlocks<T>::value)
    k_apply_a(Lats L, const typename cplx_t<T>::type *__restrict__ p, typename cplx_t<T>::type *__restrict__ t,
              double kd, double *part_t, double *part_p, int tpb, Fuse f) {
    typedef typename cplx_t<T>::type C;
    typedef TileMap<BC, NR> TM;
    const T kappa = (T)kd;
    __shared__ double sm[SmemCols<BC, NR>::N];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return; // beyond this lattice's blocks (uneven batch)
    const Geom &g = la.g;
    const C *__restrict__ U = (const C *)la.U;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const int jj = (threadIdx.x % TM::TPS) * NR;
    const size_t base = la.f0 + (size_t)cl * 12 * g.V * BC + jj;
    const int ntiles = (g.V + TM::SPB - 1) / TM::SPB;
    double at[NR], ap[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) at[r] = ap[r] = 0;
    for (int tile = blockIdx.x * tpb, tend = min(ntiles, tile + tpb); tile < tend; ++tile) {
        int s = tile * TM::SPB + threadIdx.x / TM::TPS;
        if (s >= g.V) continue;
        C acc[12][NR];
        wilson_hop_auto<T, false, BC, NR>(g, U, p + base, s, acc);
        T st[NR], sp[NR]; // per-site sums in the iteration precision, one FP64 add per site
#pragma unroll
        for (int r = 0; r < NR; ++r) st[r] = sp[r] = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            size_t o = base + ((size_t)s * 12 + c) * BC;
            C v[NR];
            Cols<C, NR>::load(p + o, v);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                sp[r] += v[r].x * v[r].x + v[r].y * v[r].y;
                v[r].x -= kappa * acc[c][r].x;
                v[r].y -= kappa * acc[c][r].y;
                st[r] += v[r].x * v[r].x + v[r].y * v[r].y;
            }
            Cols<C, NR>::store(t + o, v);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            at[r] += (double)st[r];
            ap[r] += (double)sp[r];
        }
    }
    double s1 = block_total<BC, NR>(at, sm);
    double s2 = block_total<BC, NR>(ap, sm);
    if (threadIdx.x < BC) {
        part_t[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
        part_p[(prow + blockIdx.x) * BC + threadIdx.x] = s2;
    }
    fuse_step1<BC, TM::THREADS>(f, l, part_t, part_p, prow, G, sm);
}

// r -= alpha (D_W^dag t + s0 p); partial |r|^2 (NR columns per thread)
template <typename T, int BC, int NR, bool M>
__global__ void __launch_bounds__(TileMap<BC, NR>::THREADS, MinBlocks<T>::value)
    k_apply_b(Lats L, const typename cplx_t<T>::type *__restrict__ t, const typename cplx_t<T>::type *__restrict__ p,
              typename cplx_t<T>::type *__restrict__ r, const double *__restrict__ alpha, double kd, double *part_r,
              int tpb, Fuse f) {
    typedef typename cplx_t<T>::type C;
    typedef TileMap<BC, NR> TM;
    const T kappa = (T)kd;
    __shared__ double sm[SmemCols<BC, NR>::N];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return;
    const Geom &g = la.g;
    const C *__restrict__ U = (const C *)la.U;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const double s0 = la.s0;
    const int jj = (threadIdx.x % TM::TPS) * NR, j = blockIdx.y * BC + jj;
    const size_t base = la.f0 + (size_t)cl * 12 * g.V * BC + jj;
    const int ntiles = (g.V + TM::SPB - 1) / TM::SPB;
    T a[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) a[q] = (T)alpha[j + q];
    const T sh = (T)s0;
    double ar[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) ar[q] = 0;
    for (int tile = blockIdx.x * tpb, tend = min(ntiles, tile + tpb); tile < tend; ++tile) {
        int s = tile * TM::SPB + threadIdx.x / TM::TPS;
        if (s >= g.V) continue;
        C acc[12][NR];
        wilson_hop_auto<T, true, BC, NR>(g, U, t + base, s, acc);
        T sr[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) sr[q] = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            size_t o = base + ((size_t)s * 12 + c) * BC;
            C tv[NR], pv[NR], rv[NR];
            Cols<C, NR>::load(t + o, tv);
            Cols<C, NR>::load(p + o, pv);
            Cols<C, NR>::load(r + o, rv);
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                C ap;
                ap.x = tv[q].x - kappa * acc[c][q].x + sh * pv[q].x;
                ap.y = tv[q].y - kappa * acc[c][q].y + sh * pv[q].y;
                rv[q].x -= a[q] * ap.x;
                rv[q].y -= a[q] * ap.y;
                sr[q] += rv[q].x * rv[q].x + rv[q].y * rv[q].y;
            }
            Cols<C, NR>::store(r + o, rv);
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) ar[q] += (double)sr[q];
    }
    double s1 = block_total<BC, NR>(ar, sm);
    if (threadIdx.x < BC) part_r[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
    fuse_step2<BC, TM::THREADS>(f, l, part_r, prow, G, sm);
}

// ------------------------------------------------------------------ FP32 D_W pair, neighbours staged
// k_apply_a / k_apply_b for FP32 iterations (one column per thread) with the
// neighbour sites brought into shared memory by bulk asynchronous copies
// (stage.cuh): the same arithmetic in the same order, NS stages of SPB sites
// in dynamic shared memory, *err set if a copy wait runs out.
// three 240-thread blocks per SM (<= 91 registers a thread; 3 x 71 KB of shared memory)
template <int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC>::THREADS, 3)
    k_apply_a_st(Lats L, const float2 *__restrict__ p, float2 *__restrict__ t, double kd, double *part_t,
                 double *part_p, int tpb, Fuse f, int *err) {
    typedef TileMap<BC> TM;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ double sm[SmemCols<BC, 1>::N];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return;
    const Geom &g = la.g;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const int jj = threadIdx.x % BC;
    const size_t tb = la.f0 + (size_t)cl * 12 * g.V * BC; // this RHS tile of the fields
    const int ntiles = (g.V + TM::SPB - 1) / TM::SPB;
    const int tile0 = blockIdx.x * tpb, ntb = min(ntiles, tile0 + tpb) - tile0;
    const float kappa = (float)kd;
    stage::Runner<false, BC, stage::NSTAGE> run(dsm, g, (const float2 *)la.U, p + tb, tile0, ntb, err);
    double at = 0, ap = 0;
    for (int tl = 0; tl < ntb; ++tl) {
        const int s = (tile0 + tl) * TM::SPB + threadIdx.x / BC;
        const bool valid = s < g.V;
        float2 acc[12][1];
        run.hops(tl, s, valid, acc);
        if (!valid) continue;
        float st = 0, sp = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t o = tb + ((size_t)s * 12 + c) * BC + jj;
            float2 v = p[o];
            sp += v.x * v.x + v.y * v.y;
            v.x -= kappa * acc[c][0].x;
            v.y -= kappa * acc[c][0].y;
            st += v.x * v.x + v.y * v.y;
            t[o] = v;
        }
        at += (double)st;
        ap += (double)sp;
    }
    const double s1 = block_sum<BC>(at, sm);
    const double s2 = block_sum<BC>(ap, sm);
    if (threadIdx.x < BC) {
        part_t[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
        part_p[(prow + blockIdx.x) * BC + threadIdx.x] = s2;
    }
    fuse_step1<BC, TM::THREADS>(f, l, part_t, part_p, prow, G, sm);
}

template <int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC>::THREADS, 3)
    k_apply_b_st(Lats L, const float2 *__restrict__ t, const float2 *__restrict__ p, float2 *__restrict__ r,
                 const double *__restrict__ alpha, double kd, double *part_r, int tpb, Fuse f, int *err) {
    typedef TileMap<BC> TM;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ double sm[SmemCols<BC, 1>::N];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return;
    const Geom &g = la.g;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const int jj = threadIdx.x % BC, j = blockIdx.y * BC + jj;
    const size_t tb = la.f0 + (size_t)cl * 12 * g.V * BC;
    const int ntiles = (g.V + TM::SPB - 1) / TM::SPB;
    const int tile0 = blockIdx.x * tpb, ntb = min(ntiles, tile0 + tpb) - tile0;
    const float a = (float)alpha[j], sh = (float)la.s0, kappa = (float)kd;
    stage::Runner<true, BC, stage::NSTAGE> run(dsm, g, (const float2 *)la.U, t + tb, tile0, ntb, err);
    double ar = 0;
    for (int tl = 0; tl < ntb; ++tl) {
        const int s = (tile0 + tl) * TM::SPB + threadIdx.x / BC;
        const bool valid = s < g.V;
        float2 acc[12][1];
        run.hops(tl, s, valid, acc);
        if (!valid) continue;
        float sr = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t o = tb + ((size_t)s * 12 + c) * BC + jj;
            const float2 tv = t[o], pv = p[o];
            float2 rv = r[o];
            const float apx = tv.x - kappa * acc[c][0].x + sh * pv.x;
            const float apy = tv.y - kappa * acc[c][0].y + sh * pv.y;
            rv.x -= a * apx;
            rv.y -= a * apy;
            sr += rv.x * rv.x + rv.y * rv.y;
            r[o] = rv;
        }
        ar += (double)sr;
    }
    const double s1 = block_sum<BC>(ar, sm);
    if (threadIdx.x < BC) part_r[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
    fuse_step2<BC, TM::THREADS>(f, l, part_r, prow, G, sm);
}

// The float-float pair (the first phase of SMPQ_MIXED) with staged neighbours
// and links (stage.cuh, two stages): the epilogues of k_apply_a / k_apply_b.
template <int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC>::THREADS, MinBlocks<df64>::value)
    k_apply_a_dfst(Lats L, const df64c *__restrict__ p, df64c *__restrict__ t, df64 kappa, double *part_t,
                   double *part_p, int tpb, Fuse f, int *err) {
    typedef TileMap<BC> TM;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ double sm[SmemCols<BC, 1>::N];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return;
    const Geom &g = la.g;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const int jj = threadIdx.x % BC;
    const size_t tb = la.f0 + (size_t)cl * 12 * g.V * BC;
    const int ntiles = (g.V + TM::SPB - 1) / TM::SPB;
    const int tile0 = blockIdx.x * tpb, ntb = min(ntiles, tile0 + tpb) - tile0;
    stage::RunnerDF<false, BC, stage::NSTAGE_DF> run(dsm, g, (const df64c *)la.U, p + tb, tile0, ntb, err);
    double at = 0, ap = 0;
    for (int tl = 0; tl < ntb; ++tl) {
        const int s = (tile0 + tl) * TM::SPB + threadIdx.x / BC;
        const bool valid = s < g.V;
        df64c acc[12][1];
        run.hops(tl, s, valid, acc);
        if (!valid) continue;
        df64 st = 0, sp = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t o = tb + ((size_t)s * 12 + c) * BC + jj;
            df64c v = p[o];
            sp += v.x * v.x + v.y * v.y;
            v.x -= kappa * acc[c][0].x;
            v.y -= kappa * acc[c][0].y;
            st += v.x * v.x + v.y * v.y;
            t[o] = v;
        }
        at += (double)st;
        ap += (double)sp;
    }
    const double s1 = block_sum<BC>(at, sm);
    const double s2 = block_sum<BC>(ap, sm);
    if (threadIdx.x < BC) {
        part_t[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
        part_p[(prow + blockIdx.x) * BC + threadIdx.x] = s2;
    }
    fuse_step1<BC, TM::THREADS>(f, l, part_t, part_p, prow, G, sm);
}

template <int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC>::THREADS, MinBlocks<df64>::value)
    k_apply_b_dfst(Lats L, const df64c *__restrict__ t, const df64c *__restrict__ p, df64c *__restrict__ r,
                   const double *__restrict__ alpha, df64 kappa, double *part_r, int tpb, Fuse f, int *err) {
    typedef TileMap<BC> TM;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ double sm[SmemCols<BC, 1>::N];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return;
    const Geom &g = la.g;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const int jj = threadIdx.x % BC, j = blockIdx.y * BC + jj;
    const size_t tb = la.f0 + (size_t)cl * 12 * g.V * BC;
    const int ntiles = (g.V + TM::SPB - 1) / TM::SPB;
    const int tile0 = blockIdx.x * tpb, ntb = min(ntiles, tile0 + tpb) - tile0;
    const df64 a(alpha[j]), sh(la.s0);
    stage::RunnerDF<true, BC, stage::NSTAGE_DF> run(dsm, g, (const df64c *)la.U, t + tb, tile0, ntb, err);
    double ar = 0;
    for (int tl = 0; tl < ntb; ++tl) {
        const int s = (tile0 + tl) * TM::SPB + threadIdx.x / BC;
        const bool valid = s < g.V;
        df64c acc[12][1];
        run.hops(tl, s, valid, acc);
        if (!valid) continue;
        df64 sr = 0;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t o = tb + ((size_t)s * 12 + c) * BC + jj;
            const df64c tv = t[o], pv = p[o];
            df64c rv = r[o];
            df64c apv;
            apv.x = tv.x - kappa * acc[c][0].x + sh * pv.x;
            apv.y = tv.y - kappa * acc[c][0].y + sh * pv.y;
            rv.x -= a * apv.x;
            rv.y -= a * apv.y;
            sr += rv.x * rv.x + rv.y * rv.y;
            r[o] = rv;
        }
        ar += (double)sr;
    }
    const double s1 = block_sum<BC>(ar, sm);
    if (threadIdx.x < BC) part_r[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
    fuse_step2<BC, TM::THREADS>(f, l, part_r, prow, G, sm);
}

template <int BC, bool M> cudaError_t staged_df_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    const int bytes = (int)stage::DimsDF<BC, stage::NSTAGE_DF>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_apply_a_dfst<BC, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply_b_dfst<BC, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done = e == cudaSuccess;
    return e;
}

// the dynamic shared memory of the staged pair (above the 48 KB default)
template <int BC, bool M> cudaError_t staged_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    const int bytes = (int)stage::Dims<BC, stage::NSTAGE>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_apply_a_st<BC, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply_b_st<BC, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done = e == cudaSuccess;
    return e;
}

// The base system's solution x accumulated by the p update: FP64 for the FP64
// iterations (the true-residual check), float-float for the FP64-accurate
// first phase of the mixed solve (the x_hi its FP32 phase's reliable updates
// continue from).
template <typename T> struct XAcc { typedef double2 type; };
template <> struct XAcc<df64> { typedef df64c type; };

// p = r + beta p on the lattice tiles of tile group bx; with x64, first
// x64 += alpha p, with xlo, first xlo += alpha p in T (the part of the base
// solution that the next residual replacement folds into x_hi)
// (tile0: first element of the block's RHS tile in the fields; the tile is
// blockIdx.y of the solve, so rhs j = blockIdx.y * BC + column)
template <typename T, int BC>
__device__ __forceinline__ void update_p_tiles(int bx, int V, size_t tile0,
                                               const typename cplx_t<T>::type *__restrict__ r,
                                               typename cplx_t<T>::type *__restrict__ p, const Scal &sc,
                                               typename XAcc<T>::type *__restrict__ x64,
                                               typename cplx_t<T>::type *__restrict__ xlo) {
    typedef typename cplx_t<T>::type C;
    const int jj = threadIdx.x % BC, j = blockIdx.y * BC + jj;
    if (!sc.upd_rhs[j]) return;
    const size_t base = tile0 + jj;
    const int ntiles = (V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    const T b = (T)sc.beta[j];
    const double a = sc.alpha[j];
    for (int tile = bx * TPB, tend = min(ntiles, tile + TPB); tile < tend; ++tile) {
        int s = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (s >= V) continue;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            size_t o = base + ((size_t)s * 12 + c) * BC;
            C rv = r[o], pv = p[o];
            if (xlo) {
                C xv = xlo[o];
                xv.x += (T)a * pv.x;
                xv.y += (T)a * pv.y;
                xlo[o] = xv;
            }
            if (x64) {
                if constexpr (std::is_same<T, df64>::value) {
                    df64c xv = x64[o];
                    const df64 ad(a);
                    xv.x = fma_df(ad, pv.x, xv.x);
                    xv.y = fma_df(ad, pv.y, xv.y);
                    x64[o] = xv;
                } else {
                    double2 xv = x64[o];
                    xv.x += a * to_d(pv.x);
                    xv.y += a * to_d(pv.y);
                    x64[o] = xv;
                }
            }
            pv.x = rv.x + b * pv.x;
            pv.y = rv.y + b * pv.y;
            p[o] = pv;
        }
    }
}

// ------------------------------------------------------------------ half-storage iterations
// SMPQ_FP16N / SMPQ_BF16N: the FP32 path (FP64 reliable updates, FP32 r, x_lo
// and shifted directions) with p and t -- the input and output of D_W --
// stored in the half format of half.cuh and the links in reconstruct-12 form.
// One thread per site and column (TileMap<BC>), FP32 arithmetic.
template <typename HT> struct HF {
    typename HT::h2 *v; // components, tiled like the FP32 fields
    float *n;           // norms [j / BC][V][BC]
};
template <typename HT> struct HLinks;
template <> struct HLinks<H16> { static const void *get(const smpq_ctx *c) { return c->Uh16.p; } };
template <> struct HLinks<B16> { static const void *get(const smpq_ctx *c) { return c->Ub16.p; } };

// r = p = b (p in the half format), x_lo = x_hi = 0; partial |b|^2
template <typename HT, int BC>
__global__ void __launch_bounds__(TileMap<BC>::THREADS)
    k_init_h(Geom g, Source src, float2 *r, HF<HT> p, float2 *xlo, df64c *xhi, double *part, int G) {
    __shared__ double sm[TileMap<BC>::THREADS];
    const int jj = threadIdx.x % BC, chunk = blockIdx.y, j = chunk * BC + jj;
    const size_t base = (size_t)chunk * 12 * g.V * BC + jj, nbase = (size_t)chunk * g.V * BC + jj;
    const int ntiles = (g.V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    double acc = 0;
    for (int tile = blockIdx.x * TPB, tend = min(ntiles, tile + TPB); tile < tend; ++tile) {
        const int s = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (s >= g.V) continue;
        float2 v[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t o = base + ((size_t)s * 12 + c) * BC;
            const double2 b = source_at<BC>(src, g.V, s, c, j, o);
            v[c] = make_float2((float)b.x, (float)b.y);
            r[o] = v[c];
            xlo[o] = make_float2(0.f, 0.f);
            xhi[o] = df64c{df64(0.f), df64(0.f)};
            acc += b.x * b.x + b.y * b.y;
        }
        st_site_half<HT, BC>(p.v + base + (size_t)s * 12 * BC, p.n + nbase + (size_t)s * BC, v);
    }
    const double t = block_sum<BC>(acc, sm);
    if (threadIdx.x < BC) part[((size_t)chunk * G + blockIdx.x) * BC + threadIdx.x] = t;
}

// t = D_W p in the half format; partials |t|^2 (before rounding) and |p|^2
template <typename HT, int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC>::THREADS, 3)
    k_apply_a_h(Lats L, HF<HT> p, HF<HT> t, float kappa, double *part_t, double *part_p, int tpb, Fuse f) {
    __shared__ double sm[TileMap<BC>::THREADS];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return;
    const Geom &g = la.g;
    const typename HT::h2 *__restrict__ U = (const typename HT::h2 *)la.U;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const int jj = threadIdx.x % BC;
    const size_t base = la.f0 + (size_t)cl * 12 * g.V * BC + jj, nbase = la.f0 / 12 + (size_t)cl * g.V * BC + jj;
    const int ntiles = (g.V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    double at = 0, ap = 0;
    for (int tile = blockIdx.x * tpb, tend = min(ntiles, tile + tpb); tile < tend; ++tile) {
        const int s = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (s >= g.V) continue;
        float2 acc[12][1];
        wilson_hop_half<HT, false, BC>(g, U, p.v + base, p.n + nbase, s, acc);
        const typename HT::h2 *ps = p.v + base + (size_t)s * 12 * BC;
        const float n = p.n[nbase + (size_t)s * BC];
        float sp = 0.f, st = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const float2 f = HT::f2(ps[c * BC]);
            const float2 v = make_float2(n * f.x, n * f.y);
            sp += v.x * v.x + v.y * v.y;
            acc[c][0] = make_float2(fmaf(-kappa, acc[c][0].x, v.x), fmaf(-kappa, acc[c][0].y, v.y));
            st += acc[c][0].x * acc[c][0].x + acc[c][0].y * acc[c][0].y;
        }
        float2 w[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) w[c] = acc[c][0];
        st_site_half<HT, BC>(t.v + base + (size_t)s * 12 * BC, t.n + nbase + (size_t)s * BC, w);
        at += (double)st;
        ap += (double)sp;
    }
    const double s1 = block_sum<BC>(at, sm);
    const double s2 = block_sum<BC>(ap, sm);
    if (threadIdx.x < BC) {
        part_t[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
        part_p[(prow + blockIdx.x) * BC + threadIdx.x] = s2;
    }
    fuse_step1<BC, TileMap<BC>::THREADS>(f, l, part_t, part_p, prow, G, sm);
}

// r -= alpha (D_W^dag t + s0 p); partial |r|^2
template <typename HT, int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC>::THREADS, 3)
    k_apply_b_h(Lats L, HF<HT> t, HF<HT> p, float2 *__restrict__ r, const double *__restrict__ alpha, float kappa,
                double *part_r, int tpb, Fuse f) {
    __shared__ double sm[TileMap<BC>::THREADS];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return;
    const Geom &g = la.g;
    const typename HT::h2 *__restrict__ U = (const typename HT::h2 *)la.U;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const double s0 = la.s0;
    const int jj = threadIdx.x % BC, j = blockIdx.y * BC + jj;
    const size_t base = la.f0 + (size_t)cl * 12 * g.V * BC + jj, nbase = la.f0 / 12 + (size_t)cl * g.V * BC + jj;
    const int ntiles = (g.V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    const float a = (float)alpha[j], sh = (float)s0;
    double ar = 0;
    for (int tile = blockIdx.x * tpb, tend = min(ntiles, tile + tpb); tile < tend; ++tile) {
        const int s = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (s >= g.V) continue;
        float2 acc[12][1];
        wilson_hop_half<HT, true, BC>(g, U, t.v + base, t.n + nbase, s, acc);
        const typename HT::h2 *ts = t.v + base + (size_t)s * 12 * BC, *pq = p.v + base + (size_t)s * 12 * BC;
        const float nt = t.n[nbase + (size_t)s * BC], np = p.n[nbase + (size_t)s * BC];
        float sr = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t o = base + ((size_t)s * 12 + c) * BC;
            const float2 tf = HT::f2(ts[c * BC]), pf = HT::f2(pq[c * BC]);
            const float2 pv = make_float2(np * pf.x, np * pf.y);
            float2 apv;
            apv.x = fmaf(sh, pv.x, fmaf(-kappa, acc[c][0].x, nt * tf.x));
            apv.y = fmaf(sh, pv.y, fmaf(-kappa, acc[c][0].y, nt * tf.y));
            float2 rv = r[o];
            rv.x = fmaf(-a, apv.x, rv.x);
            rv.y = fmaf(-a, apv.y, rv.y);
            r[o] = rv;
            sr += rv.x * rv.x + rv.y * rv.y;
        }
        ar += (double)sr;
    }
    const double s1 = block_sum<BC>(ar, sm);
    if (threadIdx.x < BC) part_r[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
    fuse_step2<BC, TileMap<BC>::THREADS>(f, l, part_r, prow, G, sm);
}

// p = r + beta p on the lattice tiles of tile group bx, p in the half format
template <typename HT, int BC>
__device__ __forceinline__ void update_p_h_tiles(int bx, int V, size_t tile0, const float2 *__restrict__ r,
                                                 HF<HT> p, const Scal &sc, float2 *__restrict__ xlo) {
    const int jj = threadIdx.x % BC, j = blockIdx.y * BC + jj;
    if (!sc.upd_rhs[j]) return;
    const size_t base = tile0 + jj, nbase = tile0 / 12 + jj;
    const int ntiles = (V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    const float b = (float)sc.beta[j], a = (float)sc.alpha[j];
    for (int tile = bx * TPB, tend = min(ntiles, tile + TPB); tile < tend; ++tile) {
        const int s = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (s >= V) continue;
        typename HT::h2 *ps = p.v + base + (size_t)s * 12 * BC;
        float *pn = p.n + nbase + (size_t)s * BC;
        const float n = *pn;
        float2 v[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t o = base + ((size_t)s * 12 + c) * BC;
            const float2 f = HT::f2(ps[c * BC]), rv = r[o];
            if (xlo) { // x_lo += alpha p (p as stored: n times the half value)
                float2 xv = xlo[o];
                xv.x = fmaf(a * n, f.x, xv.x);
                xv.y = fmaf(a * n, f.y, xv.y);
                xlo[o] = xv;
            }
            v[c] = make_float2(fmaf(b * n, f.x, rv.x), fmaf(b * n, f.y, rv.y));
        }
        st_site_half<HT, BC>(ps, pn, v);
    }
}

// Two columns per thread (the packed lanes of half.cuh) forms of k_apply_a_h
// and k_apply_b_h, used for even tile widths: half the FP32 instructions and
// one link reconstruction per two columns; r and x_lo move as 16-byte pairs.
template <int BC> __device__ __forceinline__ void ld_rx2(const float2 *p, float2 &re, float2 &im) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    re = make_float2(q.x, q.z);
    im = make_float2(q.y, q.w);
}
template <int BC> __device__ __forceinline__ void st_rx2(float2 *p, float2 re, float2 im) {
    *reinterpret_cast<float4 *>(p) = make_float4(re.x, im.x, re.y, im.y);
}

template <typename HT, int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC, 2>::THREADS, 2)
    k_apply_a_h2(Lats L, HF<HT> p, HF<HT> t, float kappa, double *part_t, double *part_p, int tpb, Fuse f) {
    typedef TileMap<BC, 2> TM;
    __shared__ double sm[SmemCols<BC, 2>::N];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return;
    const Geom &g = la.g;
    const typename HT::h2 *__restrict__ U = (const typename HT::h2 *)la.U;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const int jj = (threadIdx.x % TM::TPS) * 2;
    const size_t base = la.f0 + (size_t)cl * 12 * g.V * BC + jj, nbase = la.f0 / 12 + (size_t)cl * g.V * BC + jj;
    const int ntiles = (g.V + TM::SPB - 1) / TM::SPB;
    double at[2] = {0, 0}, ap[2] = {0, 0};
    const float2 nk = bc2(-kappa);
    for (int tile = blockIdx.x * tpb, tend = min(ntiles, tile + tpb); tile < tend; ++tile) {
        const int s = tile * TM::SPB + threadIdx.x / TM::TPS;
        if (s >= g.V) continue;
        c2 acc[12];
        wilson_hop_half_c2<HT, false, BC>(g, U, p.v + base, p.n + nbase, s, acc);
        const typename HT::h2 *ps = p.v + base + (size_t)s * 12 * BC;
        const float2 np = *reinterpret_cast<const float2 *>(p.n + nbase + (size_t)s * BC);
        float2 sp = bc2(0.f), st = bc2(0.f);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const c2 f = ld_c2<HT>(ps + c * BC);
            const float2 vr = __fmul2_rn(np, f.r), vi = __fmul2_rn(np, f.i);
            sp = __ffma2_rn(vr, vr, __ffma2_rn(vi, vi, sp));
            acc[c].r = __ffma2_rn(nk, acc[c].r, vr);
            acc[c].i = __ffma2_rn(nk, acc[c].i, vi);
            st = __ffma2_rn(acc[c].r, acc[c].r, __ffma2_rn(acc[c].i, acc[c].i, st));
        }
        st_site_half_c2<HT, BC>(t.v + base + (size_t)s * 12 * BC, t.n + nbase + (size_t)s * BC, acc);
        at[0] += (double)st.x;
        at[1] += (double)st.y;
        ap[0] += (double)sp.x;
        ap[1] += (double)sp.y;
    }
    const double s1 = block_total<BC, 2>(at, sm);
    const double s2 = block_total<BC, 2>(ap, sm);
    if (threadIdx.x < BC) {
        part_t[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
        part_p[(prow + blockIdx.x) * BC + threadIdx.x] = s2;
    }
    fuse_step1<BC, TM::THREADS>(f, l, part_t, part_p, prow, G, sm);
}

template <typename HT, int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC, 2>::THREADS, 2)
    k_apply_b_h2(Lats L, HF<HT> t, HF<HT> p, float2 *__restrict__ r, const double *__restrict__ alpha, float kappa,
                 double *part_r, int tpb, Fuse f) {
    typedef TileMap<BC, 2> TM;
    __shared__ double sm[SmemCols<BC, 2>::N];
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    if ((int)blockIdx.x >= la.G) return;
    const Geom &g = la.g;
    const typename HT::h2 *__restrict__ U = (const typename HT::h2 *)la.U;
    const int G = la.G, cl = blockIdx.y - la.chunk0;
    const size_t prow = la.p0 + (size_t)cl * G;
    const double s0 = la.s0;
    const int jj = (threadIdx.x % TM::TPS) * 2, j = blockIdx.y * BC + jj;
    const size_t base = la.f0 + (size_t)cl * 12 * g.V * BC + jj, nbase = la.f0 / 12 + (size_t)cl * g.V * BC + jj;
    const int ntiles = (g.V + TM::SPB - 1) / TM::SPB;
    const float2 a = make_float2((float)alpha[j], (float)alpha[j + 1]), na = make_float2(-a.x, -a.y);
    const float2 sh = bc2((float)s0), nk = bc2(-kappa);
    double ar[2] = {0, 0};
    for (int tile = blockIdx.x * tpb, tend = min(ntiles, tile + tpb); tile < tend; ++tile) {
        const int s = tile * TM::SPB + threadIdx.x / TM::TPS;
        if (s >= g.V) continue;
        c2 acc[12];
        wilson_hop_half_c2<HT, true, BC>(g, U, t.v + base, t.n + nbase, s, acc);
        const typename HT::h2 *ts = t.v + base + (size_t)s * 12 * BC, *pq = p.v + base + (size_t)s * 12 * BC;
        const float2 nt = *reinterpret_cast<const float2 *>(t.n + nbase + (size_t)s * BC);
        const float2 np = *reinterpret_cast<const float2 *>(p.n + nbase + (size_t)s * BC);
        float2 sr = bc2(0.f);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const size_t o = base + ((size_t)s * 12 + c) * BC;
            const c2 tf = ld_c2<HT>(ts + c * BC), pf = ld_c2<HT>(pq + c * BC);
            const float2 pr = __fmul2_rn(np, pf.r), pi = __fmul2_rn(np, pf.i);
            // A p = D_W^dag t + s0 p
            const float2 apr = __ffma2_rn(sh, pr, __ffma2_rn(nk, acc[c].r, __fmul2_rn(nt, tf.r)));
            const float2 api = __ffma2_rn(sh, pi, __ffma2_rn(nk, acc[c].i, __fmul2_rn(nt, tf.i)));
            float2 rr, ri;
            ld_rx2<BC>(r + o, rr, ri);
            rr = __ffma2_rn(na, apr, rr);
            ri = __ffma2_rn(na, api, ri);
            st_rx2<BC>(r + o, rr, ri);
            sr = __ffma2_rn(rr, rr, __ffma2_rn(ri, ri, sr));
        }
        ar[0] += (double)sr.x;
        ar[1] += (double)sr.y;
    }
    const double s1 = block_total<BC, 2>(ar, sm);
    if (threadIdx.x < BC) part_r[(prow + blockIdx.x) * BC + threadIdx.x] = s1;
    fuse_step2<BC, TM::THREADS>(f, l, part_r, prow, G, sm);
}

// Shifted updates on the support: y += c_i alpha_i p_i ; p_i = zeta_new_i r + beta_i p_i.
// Support entry k of rhs j sits on lattice site supsite[rhs_class[j] * n_sup + k]
// (identity when supsite == nullptr).  r is read in the iteration precision T,
// ps ([shift][chunk][n_sup][12][BC]) is kept in TS, y ([chunk][n_sup][12][BC]) in FP64.
// (one lattice: rtile0 is the first element of the RHS tile in r, cl the tile
// within the lattice, j0 the solve's first rhs of the tile; ps and y are the
// lattice's support fields, [shift][tile][n_sup][12][BC] and
// [tile][n_sup][12][BC] for its B right-hand sides; the shift-major scalars
// have stride Btot)
template <typename T, typename TS, int BC>
__device__ __forceinline__ void shift_tiles(int bx, int cl, int j0, size_t rtile0, int n_sup, int nshift, int B,
                                            int Btot, const int *__restrict__ supsite,
                                            const int *__restrict__ rhs_class,
                                            const typename cplx_t<T>::type *__restrict__ r,
                                            typename cplx_t<TS>::type *__restrict__ ps, double2 *__restrict__ y,
                                            const Scal &sc, const ShiftParams &sp, int init) {
    typedef typename cplx_t<T>::type CR;
    typedef typename cplx_t<TS>::type C;
    const int jj = threadIdx.x % BC, j = j0 + jj;
    const int cls = rhs_class[j];
    if (cls < 0) return;
    const size_t rbase = rtile0 + jj;
    const size_t sbase = (size_t)cl * 12 * n_sup * BC + jj;
    const size_t sstride = (size_t)B * 12 * n_sup; // one shift
    const int ntiles = (n_sup + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    for (int tile = bx * TPB, tend = min(ntiles, tile + TPB); tile < tend; ++tile) {
        int k = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (k >= n_sup) continue;
        int site = supsite ? supsite[(size_t)cls * n_sup + k] : k;
        C rv[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            CR v = r[rbase + ((size_t)site * 12 + c) * BC];
            rv[c] = mkc<C>(to_d(v.x), to_d(v.y));
        }
        if (init) { // p_i = b (= r at the start), y = 0
            for (int i = 0; i < nshift; ++i)
#pragma unroll
                for (int c = 0; c < 12; ++c) ps[i * sstride + sbase + ((size_t)k * 12 + c) * BC] = rv[c];
#pragma unroll
            for (int c = 0; c < 12; ++c) y[sbase + ((size_t)k * 12 + c) * BC] = make_double2(0, 0);
            continue;
        }
        double2 yv[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) yv[c] = y[sbase + ((size_t)k * 12 + c) * BC];
        for (int i = 0; i < nshift; ++i) {
            if (!sc.upd[i * Btot + j]) continue;
            double ca = sp.c[i] * sc.alpha_s[i * Btot + j];
            TS zn = (TS)sc.zeta_new[i * Btot + j];
            TS bs = (TS)sc.beta_s[i * Btot + j];
            C *pi = ps + i * sstride + sbase;
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                size_t o = ((size_t)k * 12 + c) * BC;
                C pv = pi[o];
                yv[c].x += ca * (double)pv.x;
                yv[c].y += ca * (double)pv.y;
                pv.x = zn * rv[c].x + bs * pv.x;
                pv.y = zn * rv[c].y + bs * pv.y;
                pi[o] = pv;
            }
        }
#pragma unroll
        for (int c = 0; c < 12; ++c) y[sbase + ((size_t)k * 12 + c) * BC] = yv[c];
    }
}

// shifted directions at the start of a solve: p_i = b (= r), y = 0
// (one lattice per launch: blockIdx.y is its tile, chunk0 its first tile in
// the solve; r points at the lattice's part of the field)
template <typename T, typename TS, int BC>
__global__ void __launch_bounds__(TileMap<BC>::THREADS)
    k_shift_init(int V, int n_sup, int nshift, int B, int chunk0, const int *__restrict__ supsite,
                 const int *__restrict__ rhs_class, const typename cplx_t<T>::type *__restrict__ r,
                 typename cplx_t<TS>::type *__restrict__ ps, double2 *__restrict__ y, Scal sc, ShiftParams sp) {
    shift_tiles<T, TS, BC>(blockIdx.x, blockIdx.y, (chunk0 + blockIdx.y) * BC, (size_t)blockIdx.y * 12 * V * BC, n_sup,
                           nshift, B, B, supsite, rhs_class, r, ps, y, sc, sp, 1);
}

// Launch YP of an iteration: blocks x < Gs update y and the shifted directions
// on the support, the others p (and x64) on the lattice.
template <typename T, typename TS, int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC>::THREADS)
    k_yp(Lats L, int nshift, int Btot, const int *__restrict__ rhs_class, const typename cplx_t<T>::type *__restrict__ r,
         typename cplx_t<TS>::type *__restrict__ ps, double2 *__restrict__ y, Scal sc,
         const ShiftParams *__restrict__ sp, typename cplx_t<T>::type *__restrict__ p,
         typename XAcc<T>::type *__restrict__ x64, typename cplx_t<T>::type *__restrict__ xlo) {
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    const int cl = blockIdx.y - la.chunk0, bx = blockIdx.x;
    const size_t tile0 = la.f0 + (size_t)cl * 12 * la.g.V * BC;
    if (bx < la.Gs)
        shift_tiles<T, TS, BC>(bx, cl, blockIdx.y * BC, tile0, la.n_sup, nshift, la.B, Btot, la.supsite, rhs_class, r,
                               ps + (size_t)nshift * la.sup0, y + la.sup0, sc, sp[l], 0);
    else if (bx < la.Gs + la.G)
        update_p_tiles<T, BC>(bx - la.Gs, la.g.V, tile0, r, p, sc, x64, xlo);
}

// Launch YP of a half-storage iteration (p in the half format)
template <typename HT, int BC, bool M>
__global__ void __launch_bounds__(TileMap<BC>::THREADS)
    k_yp_h(Lats L, int nshift, int Btot, const int *__restrict__ rhs_class, const float2 *__restrict__ r,
           float2 *__restrict__ ps, double2 *__restrict__ y, Scal sc, const ShiftParams *__restrict__ sp, HF<HT> p,
           float2 *__restrict__ xlo) {
    const int l = lat_index<M>(L);
    const Lat &la = L.l[l];
    const int cl = blockIdx.y - la.chunk0, bx = blockIdx.x;
    const size_t tile0 = la.f0 + (size_t)cl * 12 * la.g.V * BC;
    if (bx < la.Gs)
        shift_tiles<float, float, BC>(bx, cl, blockIdx.y * BC, tile0, la.n_sup, nshift, la.B, Btot, la.supsite,
                                      rhs_class, r, ps + (size_t)nshift * la.sup0, y + la.sup0, sc, sp[l], 0);
    else if (bx < la.Gs + la.G)
        update_p_h_tiles<HT, BC>(bx - la.Gs, la.g.V, tile0, r, p, sc, xlo);
}

// x_hi += x_lo ; x_lo = 0 (x_hi in float-float: FP64 accuracy on the FP32 pipes)
template <typename T, int BC>
__global__ void __launch_bounds__(TileMap<BC>::THREADS)
    k_rel_accum(int V, df64c *__restrict__ xhi, typename cplx_t<T>::type *__restrict__ xlo, int G) {
    typedef typename cplx_t<T>::type C;
    const int jj = threadIdx.x % BC, chunk = blockIdx.y;
    const size_t base = (size_t)chunk * 12 * V * BC + jj;
    const int ntiles = (V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    for (int tile = blockIdx.x * TPB, tend = min(ntiles, tile + TPB); tile < tend; ++tile) {
        int s = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (s >= V) continue;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            size_t o = base + ((size_t)s * 12 + c) * BC;
            C xl = xlo[o];
            df64c xh = xhi[o];
            xh.x = xh.x + df64(xl.x);
            xh.y = xh.y + df64(xl.y);
            xhi[o] = xh;
            xlo[o] = mkc<C>(0, 0);
        }
    }
}

// r_hi = b - (D_W^dag t64 + s0 x_hi) in FP64 (t64 = D_W x_hi); r = T(r_hi); partial |r_hi|^2
template <typename T, int BC>
__global__ void __launch_bounds__(TileMap<BC>::THREADS)
    k_rel_resid(Geom g, const double2 *__restrict__ U64, const double2 *__restrict__ t64,
                const double2 *__restrict__ xhi, Source src, typename cplx_t<T>::type *__restrict__ r, double s0,
                double kappa, double *part_r, int G) {
    typedef typename cplx_t<T>::type C;
    __shared__ double sm[TileMap<BC>::THREADS];
    const int jj = threadIdx.x % BC, chunk = blockIdx.y, j = chunk * BC + jj;
    const size_t base = (size_t)chunk * 12 * g.V * BC + jj;
    const int ntiles = (g.V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    double ar = 0;
    for (int tile = blockIdx.x * TPB, tend = min(ntiles, tile + TPB); tile < tend; ++tile) {
        int s = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (s >= g.V) continue;
        double2 acc[12][1];
        wilson_hop<double, true, BC>(g, U64, t64 + base, s, acc);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            size_t o = base + ((size_t)s * 12 + c) * BC;
            double2 tv = t64[o], xv = xhi[o];
            double2 b = source_at<BC>(src, g.V, s, c, j, o);
            double2 rv;
            rv.x = b.x - (tv.x - kappa * acc[c][0].x + s0 * xv.x);
            rv.y = b.y - (tv.y - kappa * acc[c][0].y + s0 * xv.y);
            r[o] = mkc<C>(rv.x, rv.y);
            ar += rv.x * rv.x + rv.y * rv.y;
        }
    }
    double s1 = block_sum<BC>(ar, sm);
    if (threadIdx.x < BC) part_r[((size_t)chunk * G + blockIdx.x) * BC + threadIdx.x] = s1;
}

// Residual replacement in float-float (FP64-accurate, on the FP32 pipes):
// r_hi = b - (D_W^dag t + s0 x_hi) with t = D_W x_hi (both float-float fields);
// r = T(r_hi); partial |r_hi|^2 (per-site sums of the high parts in FP32: the
// norm only steers the recurrences and the convergence test).
template <typename T, int BC>
__global__ void __launch_bounds__(TileMap<BC>::THREADS, MinBlocks<df64>::value)
    k_rel_resid_df(Geom g, const df64c *__restrict__ U, const df64c *__restrict__ t, const df64c *__restrict__ xhi,
                   Source src, typename cplx_t<T>::type *__restrict__ r, double s0, df64 kappa, double *part_r,
                   int G) {
    typedef typename cplx_t<T>::type C;
    __shared__ double sm[TileMap<BC>::THREADS];
    const int jj = threadIdx.x % BC, chunk = blockIdx.y, j = chunk * BC + jj;
    const size_t base = (size_t)chunk * 12 * g.V * BC + jj;
    const int ntiles = (g.V + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
    const df64 sh(s0);
    const int cls = src.b64 ? -1 : src.src_class[j], comp = src.b64 ? -1 : src.src_comp[j];
    double ar = 0;
    for (int tile = blockIdx.x * TPB, tend = min(ntiles, tile + TPB); tile < tend; ++tile) {
        int s = tile * TileMap<BC>::SPB + threadIdx.x / BC;
        if (s >= g.V) continue;
        df64c acc[12][1];
        wilson_hop_auto<df64, true, BC>(g, U, t + base, s, acc);
        const bool in_class = cls >= 0 && src.colour[s] == cls;
        float sr = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            size_t o = base + ((size_t)s * 12 + c) * BC;
            const df64c tv = t[o], xv = xhi[o];
            df64c bv;
            if (src.b64) bv = df64c{df64(src.b64[o].x), df64(src.b64[o].y)}; // explicit source (rare)
            else bv = df64c{df64((in_class && c == comp) ? 1.f : 0.f), df64(0.f)};
            df64c rv;
            rv.x = bv.x - (tv.x - kappa * acc[c][0].x + sh * xv.x);
            rv.y = bv.y - (tv.y - kappa * acc[c][0].y + sh * xv.y);
            if constexpr (std::is_same<T, float>::value) r[o] = make_float2(rv.x.hi + rv.x.lo, rv.y.hi + rv.y.lo);
            else if constexpr (std::is_same<T, df64>::value) r[o] = rv;
            else r[o] = mkc<C>(to_d(rv.x), to_d(rv.y));
            sr += rv.x.hi * rv.x.hi + rv.y.hi * rv.y.hi;
        }
        ar += (double)sr;
    }
    double s1 = block_sum<BC>(ar, sm);
    if (threadIdx.x < BC) part_r[((size_t)chunk * G + blockIdx.x) * BC + threadIdx.x] = s1;
}

// ------------------------------------------------------------------ scalar kernels (one block per rhs)
constexpr int SCAL_THREADS = 128;

// sum over blocks of the partials of rhs j: strided per-thread sums, then a
// fixed tree (deterministic)
__device__ __forceinline__ double part_sum(const double *part, int j, int BC, int G, double *sm) {
    const int chunk = j / BC, jj = j % BC;
    double s = 0;
    for (int b = threadIdx.x; b < G; b += SCAL_THREADS) s += part[((size_t)chunk * G + b) * BC + jj];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int st = SCAL_THREADS / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
        __syncthreads();
    }
    double r = sm[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAL_THREADS)
    s_init(int B, int BC, int G, const double *part_b, Scal sc, ShiftParams sp, double tol) {
    __shared__ double sm[SCAL_THREADS];
    const int j = blockIdx.x;
    double bb = part_sum(part_b, j, BC, G, sm);
    if (threadIdx.x) return;
    sc.bb[j] = bb;
    sc.rr[j] = bb;
    sc.rr_ref[j] = bb;
    sc.alpha[j] = 0;
    sc.beta[j] = 0;
    sc.alpha_prev[j] = 1;
    sc.beta_prev[j] = 0;
    sc.iters[j] = 0;
    int any = 0;
    for (int i = 0; i < sp.n; ++i) {
        sc.zeta[i * B + j] = 1;
        sc.zeta_prev[i * B + j] = 1;
        sc.zeta_new[i * B + j] = 1;
        sc.alpha_s[i * B + j] = 0;
        sc.beta_s[i * B + j] = 0;
        sc.upd[i * B + j] = 0;
        int a = bb > 0;
        sc.act[i * B + j] = a;
        any |= a;
    }
    sc.act_rhs[j] = any;
    sc.upd_rhs[j] = 0;
    if (any) atomicAdd(&sc.flags[0], 1);
}

// out[j] = sum over the blocks of the partials of rhs j (one block per rhs)
__global__ void __launch_bounds__(SCAL_THREADS) s_sum_rhs(int BC, int G, const double *part, double *out) {
    __shared__ double sm[SCAL_THREADS];
    const double v = part_sum(part, blockIdx.x, BC, G, sm);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// after a residual replacement: rr = |r_hi|^2, the base shift re-activates if
// its true residual is above tolerance (flags[0] and flags[1] are cleared by
// the host before the launch)
__global__ void __launch_bounds__(SCAL_THREADS)
    s_rel(int B, int BC, int G, const double *part_r, Scal sc, ShiftParams sp, double tol2, int base) {
    __shared__ double sm[SCAL_THREADS];
    const int j = blockIdx.x;
    double rr = part_sum(part_r, j, BC, G, sm);
    if (threadIdx.x || !(sc.bb[j] > 0)) return;
    sc.rr[j] = rr;
    sc.rr_ref[j] = rr;
    int any = 0;
    for (int i = 0; i < sp.n; ++i) {
        int ix = i * B + j;
        if (i == base) sc.act[ix] = sc.zeta[ix] * sc.zeta[ix] * rr > tol2 * sc.bb[j];
        any |= sc.act[ix];
    }
    sc.act_rhs[j] = any;
    if (any) atomicAdd(&sc.flags[0], 1);
}

// ------------------------------------------------------------------ driver

// p = r for every right-hand side whose base shift a residual replacement has
// re-activated (a restart of its CG from the true residual)
template <typename C>
__global__ void k_restart_p(const C *__restrict__ r, C *__restrict__ p, size_t n, int BC, int V,
                            const int *__restrict__ act_rhs) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = (int)(i / ((size_t)12 * V * BC)) * BC + (int)(i % BC); // tile layout [j/BC][V][12][BC]
    if (act_rhs[j]) p[i] = r[i];
}

// elementwise float-float -> FP32 copy of a field (same tiled layout)
__global__ void k_to_fp32(const df64c *__restrict__ in, float2 *__restrict__ out, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void k_d2f(const double2 *__restrict__ in, float2 *__restrict__ out, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// The second phase of SMPQ_MIXED keeps the shifted directions in FP32: their
// updates after the switch only add terms of the size of the (already small)
// residual, like the FP32 base vectors.  SMPQ_PS64 keeps them in FP64.
#ifdef SMPQ_PS64
constexpr bool ps32_phase2 = false;
#else
constexpr bool ps32_phase2 = true;
#endif

// One lattice of a solve, as its caller describes it: the context (geometry,
// links), the right-hand sides and support (spec), its rational's shifts and
// where the results go.  A solve of several lattices (the uneven batch) takes
// precision, tolerance and options from the first lattice's context.
struct LatIn {
    smpq_ctx *ctx;
    const SolveSpec *spec;
    ShiftParams sp;
    SolveOut *out;
};

// One multi-shift solve of B right-hand sides in tiles of BC columns, over
// one lattice or several of different sizes in the same launches.  The
// solve runs in one or two phases:
//   SMPQ_FP64  : FP64 iterations (vectors, D_W, shifted directions);
//   SMPQ_FP32  : FP32 iterations with FP64 reliable updates of the base system;
//   SMPQ_FP16N / SMPQ_BF16N : the same with p and t stored in FP16 / BF16 with
//                per-site norms and reconstruct-12 links;
//   SMPQ_MIXED : FP64-accurate iterations until every right-hand side has
//                ||r|| <= theta ||b||, then FP32 iterations ending in one
//                residual replacement of the base system; the shifted
//                directions are FP64 in the first phase and FP32 in the
//                second, y stays FP64 throughout.
// Scalars, reductions and y are FP64 in every mode.  The fields of all
// lattices share one buffer per vector: lattice l's part starts at element
// f0[l] (its tiles first come at tile ch0[l] of the solve).
template <int BC> struct Solve {
    smpq_ctx *ctx; // the first lattice's context: stream, workspace, options
    std::vector<LatIn> in;
    int nl;
    // per lattice: sites, right-hand sides, tiles, first tile, first rhs, blocks
    // per tile of the one-column lattice kernels (TPB tiles each), of the
    // support kernels, one-column tiles; field, support-field and partial-row offsets
    std::vector<int> V, Bl, nch, ch0, j0, G1, Gs1, nt1;
    std::vector<size_t> f0, s0, p0;
    std::vector<Source> srcl;
    std::vector<ShiftParams> sph; // host copies behind spd
    int B = 0, nchunk = 0, nshift = 0;
    size_t nfield = 0, nsupf = 0, npart = 0;
    cudaStream_t st;
    Scal sc;
    const ShiftParams *spd = nullptr; // [nl] device copies
    double *part0, *part1, *part2;
    double2 *y;
    double tol2;
    int *hflags = nullptr;
    int *count = nullptr;       // [nchunk] arrival counters of the fused scalar steps
    double2 *x64 = nullptr;     // base-system solution in FP64 (true residual), nullable
    double *true_rr = nullptr;  // [B] |b - (A + s0) x64|^2
    int iters = 0, nrel = 0;
    bool prof;
    int chk;
    bool shifts;
    int tpb_hi = TPB, tpb_lo = TPB, nr = 1;
    bool stg = false;    // FP32 iterations: the D_W pair with staged neighbours (stage.cuh)
    bool stg_df = false; // float-float iterations: likewise

    explicit Solve(const std::vector<LatIn> &lats) : ctx(lats[0].ctx), in(lats), nl((int)lats.size()) {}

    // the per-rhs scalars of lattice l (the shift-major ones keep the solve's stride B)
    Scal scal_of(int l) const {
        Scal s = sc;
        const int o = j0[l];
        s.rr += o; s.bb += o; s.alpha += o; s.beta += o; s.alpha_prev += o; s.beta_prev += o; s.rr_ref += o;
        s.act_rhs += o; s.upd_rhs += o; s.iters += o;
        s.zeta += o; s.zeta_prev += o; s.zeta_new += o; s.alpha_s += o; s.beta_s += o; s.act += o; s.upd += o;
        return s;
    }

    int setup(double tol, double *hist, int hist_len) {
        st = ctx->stream;
        shifts = in[0].spec->n_sup > 0;
        nshift = in[0].sp.n;
        V.resize(nl); Bl.resize(nl); nch.resize(nl); ch0.resize(nl); j0.resize(nl); G1.resize(nl); Gs1.resize(nl);
        nt1.resize(nl); f0.resize(nl); s0.resize(nl); p0.resize(nl); srcl.resize(nl); sph.resize(nl);
        for (int l = 0; l < nl; ++l) {
            const SolveSpec &sp = *in[l].spec;
            if (sp.B % BC || in[l].sp.n != nshift || (sp.n_sup > 0) != shifts || in[l].ctx->device != ctx->device)
                return set_err(ctx, SMPQ_EINVAL, "lattices of one solve need the same tile width, poles, support "
                                                 "kind and device");
            V[l] = in[l].ctx->V;
            Bl[l] = sp.B;
            nch[l] = sp.B / BC;
            ch0[l] = nchunk;
            j0[l] = B;
            nt1[l] = (V[l] + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
            G1[l] = (nt1[l] + TPB - 1) / TPB;
            const int nsup_tiles = (sp.n_sup + TileMap<BC>::SPB - 1) / TileMap<BC>::SPB;
            Gs1[l] = std::max(1, (nsup_tiles + TPB - 1) / TPB);
            f0[l] = nfield;
            s0[l] = nsupf;
            p0[l] = npart / BC;
            nchunk += nch[l];
            B += sp.B;
            nfield += (size_t)sp.B * 12 * V[l];
            nsupf += (size_t)sp.B * 12 * sp.n_sup;
            // partial rows per tile: the most blocks any launch has per tile (the
            // D_W launches at one tile per block have nt1; the support kernels Gs1)
            npart += (size_t)nch[l] * std::max(nt1[l], Gs1[l]) * BC;
            sph[l] = in[l].sp;
        }
        tpb_hi = std::max(1, in[0].spec->tpb_hi > 0 ? in[0].spec->tpb_hi : TPB);
        tpb_lo = std::max(1, in[0].spec->tpb_lo > 0 ? in[0].spec->tpb_lo : TPB);
        nr = in[0].spec->nr == 2 ? 2 : 1;
        stg = (in[0].spec->staged & 1) && BC >= 12; // (one-column tiles: plain loads)
        stg_df = (in[0].spec->staged & 2) && BC >= 12;
        if (stg && nr == 2) return set_err(ctx, SMPQ_EINVAL, "internal: the staged D_W has one column per thread");
        std::vector<Buf> &ws = ctx->ws;
        if (ws.size() < W_COUNT) ws.resize(W_COUNT);
        int rc;
        if ((rc = ensure(ctx, ws[W_PART], 3 * npart * sizeof(double)))) return rc;
        const size_t nscal = (size_t)B * 8 + (size_t)nshift * B * 5;
        const size_t nint = (size_t)B * 3 + (size_t)nshift * B * 2 + 12 + (size_t)nchunk;
        const size_t spbytes = ((size_t)nl * sizeof(ShiftParams) + 255) / 256 * 256;
        if ((rc = ensure(ctx, ws[W_SCAL], spbytes + nscal * sizeof(double) + nint * sizeof(int)))) return rc;
        part0 = (double *)ws[W_PART].p;
        part1 = part0 + npart;
        part2 = part1 + npart;
        spd = (const ShiftParams *)ws[W_SCAL].p;
        cudaMemcpyAsync((void *)spd, sph.data(), nl * sizeof(ShiftParams), cudaMemcpyHostToDevice, st);
        double *d = (double *)((char *)ws[W_SCAL].p + spbytes);
        sc.rr = d; d += B; sc.bb = d; d += B; sc.alpha = d; d += B; sc.beta = d; d += B;
        sc.alpha_prev = d; d += B; sc.beta_prev = d; d += B; sc.rr_ref = d; d += B;
        sc.zeta = d; d += nshift * B; sc.zeta_prev = d; d += nshift * B; sc.zeta_new = d; d += nshift * B;
        sc.alpha_s = d; d += nshift * B; sc.beta_s = d; d += nshift * B;
        true_rr = d; d += B;
        int *ip = (int *)d;
        sc.act_rhs = ip; ip += B; sc.upd_rhs = ip; ip += B; sc.iters = ip; ip += B;
        sc.act = ip; ip += nshift * B; sc.upd = ip; ip += nshift * B;
        sc.flags = ip; ip += 8; sc.iter_counter = ip; ip += 4;
        count = ip;
        sc.hist = hist;
        sc.hist_len = hist_len;
        for (int l = 0; l < nl; ++l) { // the lattice's sources, its per-rhs tables at its first rhs
            const SolveSpec &sp = *in[l].spec;
            srcl[l].colour = sp.d_colour;
            srcl[l].src_class = sp.d_src_class ? sp.d_src_class + j0[l] : nullptr;
            srcl[l].src_comp = sp.d_src_comp ? sp.d_src_comp + j0[l] : nullptr;
            srcl[l].b64 = sp.d_src_field ? (const double2 *)sp.d_src_field + f0[l] : nullptr;
        }
        tol2 = tol * tol;
        prof = ctx->opt.profile != 0;
        chk = std::max(1, ctx->opt.iters_per_check);
        if (prof) {
            while ((int)ctx->prof_ev.size() < 4 * chk) {
                cudaEvent_t ev;
                if (cudaEventCreate(&ev) != cudaSuccess) return cuda_check(ctx, cudaGetLastError(), "event");
                ctx->prof_ev.push_back(ev);
            }
        }
        if (cudaMallocHost(&hflags, NFLAGS * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(ctx, SMPQ_ENOMEM, "pinned host flags");
        }
        cudaMemsetAsync(sc.flags, 0, (12 + (size_t)nchunk) * sizeof(int), st); // flags, counter, arrivals
        return SMPQ_OK;
    }

    ~Solve() {
        if (hflags) cudaFreeHost(hflags);
    }

    // The lattice table of a D_W launch: blocks per tile for spb sites per tile
    // and tpb tiles per block; partial rows lattice after lattice.  *gx: the
    // grid's x extent (the largest lattice's blocks).
    template <typename T, typename HT = void> Lats lats_dw(int spb, int tpb, int *gx) const {
        Lats L{};
        L.n = nl;
        size_t prow = 0;
        *gx = 1;
        for (int l = 0; l < nl; ++l) {
            Lat &a = L.l[l];
            a.g = in[l].ctx->geom;
            if constexpr (std::is_void<HT>::value) a.U = Links<T>::get(in[l].ctx);
            else a.U = HLinks<HT>::get(in[l].ctx);
            a.f0 = (long long)f0[l];
            a.chunk0 = ch0[l];
            a.G = ((V[l] + spb - 1) / spb + tpb - 1) / tpb;
            a.p0 = (long long)prow;
            a.s0 = sph[l].s0;
            a.B = Bl[l];
            prow += (size_t)nch[l] * a.G;
            *gx = std::max(*gx, a.G);
        }
        return L;
    }
    // the lattice table of launch YP: support blocks, then lattice blocks (one column, TPB tiles)
    Lats lats_yp(int *gx) const {
        Lats L{};
        L.n = nl;
        *gx = 1;
        for (int l = 0; l < nl; ++l) {
            Lat &a = L.l[l];
            a.g = in[l].ctx->geom;
            a.f0 = (long long)f0[l];
            a.chunk0 = ch0[l];
            a.G = G1[l];
            a.Gs = shifts ? Gs1[l] : 0;
            a.n_sup = in[l].spec->n_sup;
            a.supsite = in[l].spec->d_supsite;
            a.sup0 = (long long)s0[l];
            a.B = Bl[l];
            a.s0 = sph[l].s0;
            *gx = std::max(*gx, a.Gs + a.G);
        }
        return L;
    }
    // one lattice alone (its part of every buffer), for the per-lattice launches
    template <typename T> Lats lats_one(int l) const {
        Lats L{};
        L.n = 1;
        Lat &a = L.l[0];
        a.g = in[l].ctx->geom;
        a.U = Links<T>::get(in[l].ctx);
        a.f0 = (long long)f0[l];
        a.chunk0 = 0;
        a.G = G1[l];
        a.p0 = (long long)p0[l];
        a.s0 = sph[l].s0;
        a.B = Bl[l];
        return L;
    }

    void collect(int n, bool hi) {
        if (!prof) return;
        for (int k = 0; k < n; ++k) {
            float a = 0, b = 0;
            if (cudaEventElapsedTime(&a, ctx->prof_ev[4 * k], ctx->prof_ev[4 * k + 1]) != cudaSuccess ||
                cudaEventElapsedTime(&b, ctx->prof_ev[4 * k + 2], ctx->prof_ev[4 * k + 3]) != cudaSuccess) {
                cudaGetLastError();
                a = b = 0;
            }
            (hi ? ctx->prof_a_hi_ms : ctx->prof_a_ms) += a;
            (hi ? ctx->prof_b_hi_ms : ctx->prof_b_ms) += b;
        }
        (hi ? ctx->prof_a_hi_n : ctx->prof_a_n) += n;
        (hi ? ctx->prof_b_hi_n : ctx->prof_b_n) += n;
    }

    // a half-format field of this solve passed through a float2 pointer
    template <typename HT> HF<HT> hfield(void *f) const {
        typename HT::h2 *v = (typename HT::h2 *)f;
        return HF<HT>{v, (float *)(v + nfield)};
    }

    // Iterate with vectors of precision T and shifted directions of precision TS.
    // init: start from x = 0 (sources); otherwise continue from the current state.
    // rel: FP64 reliable updates (needs xlo, xhi, t64).  theta2 > 0: return once
    // every active right-hand side has ||r||^2 <= theta2 ||b||^2.
    // fixed > 0: exactly `fixed` iterations, no checks (Lanczos).
    // HT (H16 or B16, T = float): p and t are half-format fields (components,
    // then norms) passed through the float2 pointers.
    // xacc (nullable): the base solution accumulated by the p updates (FP64 for
    // FP64 iterations, float-float for the mixed solve's first phase).
    template <typename T, typename TS, typename HT = void>
    int phase(typename cplx_t<T>::type *p, typename cplx_t<T>::type *t, typename cplx_t<T>::type *r,
              typename cplx_t<T>::type *xlo, df64c *xhi, df64c *t64, typename cplx_t<TS>::type *ps, bool init,
              bool rel, double theta2, int fixed, int max_iter, typename XAcc<T>::type *xacc = nullptr,
              bool replace_mid = true) {
        typedef typename cplx_t<T>::type C;
        constexpr bool half = !std::is_void<HT>::value;
        const int TH = TileMap<BC>::THREADS;
        const bool hi = sizeof(T) != sizeof(float); // FP64 or float-float iterations
        const bool multi = nl > 1;
        // kernel shape of the D_W launches (the autotuner's choice): tiles per
        // block, per phase, and for the FP32 kernels one or two columns per thread
        const int tpb = hi ? tpb_hi : tpb_lo;
        const bool two_cols = std::is_same<T, float>::value && !half && nr == 2 && BC % 2 == 0 && !multi;
        constexpr bool can_stage = std::is_same<T, float>::value && !half && BC >= 12;
        constexpr bool can_stage_df = std::is_same<T, df64>::value && BC >= 12;
        const bool staged = can_stage && stg;
        const bool staged_df = can_stage_df && stg_df;
        if constexpr (can_stage) {
            if (staged) { // before any capture: the kernels' shared-memory limit
                const cudaError_t e = multi ? staged_attrs<BC, true>() : staged_attrs<BC, false>();
                if (e != cudaSuccess) return cuda_check(ctx, e, "staged D_W attributes");
            }
        }
        if constexpr (can_stage_df) {
            if (staged_df) {
                const cudaError_t e = multi ? staged_df_attrs<BC, true>() : staged_df_attrs<BC, false>();
                if (e != cudaSuccess) return cuda_check(ctx, e, "staged D_W attributes");
            }
        }
        // Half-storage iterations replace the residual at least every 10x drop:
        // their iterated residual drifts from the true one by about the format's
        // rounding times the condition number per iteration, so a 1000x drop
        // (the FP32 default) would outlast its meaning.
        const double delta = half ? std::max(ctx->opt.reliable_delta, 0.1) : ctx->opt.reliable_delta;
        // replace_mid = false: one replacement when every shift has converged
        // (then only the base shift can re-activate, so the replacement never
        // enters the shifted systems; the mixed solve's FP32 phase)
        const double delta2 = rel && replace_mid ? delta * delta : 0.0;
        const T kappa = (T)ctx->opt.kappa;
        const double kd = ctx->opt.kappa;
        const int per_iter = 3;
        if constexpr (half) {
            if (!rel || !xlo || !xhi || !t64)
                return set_err(ctx, SMPQ_EINVAL, "internal: half-storage iterations need FP64 reliable updates");
        }
        // every launch's partial rows must fit the partial buffers (npart per
        // buffer): the D_W launches at this tpb (one column: the most blocks)
        // and the one-column lattice kernels
        {
            size_t rows = 0;
            for (int l = 0; l < nl; ++l)
                rows += (size_t)nch[l] * std::max((nt1[l] + tpb - 1) / tpb, G1[l]);
            if (rows * BC > npart)
                return set_err(ctx, SMPQ_EINVAL, "internal: launch shape exceeds the partial-sum buffers");
        }
        if (init) {
            for (int l = 0; l < nl; ++l) {
                const dim3 grid(G1[l], nch[l]);
                const Geom &g = in[l].ctx->geom;
                const size_t o = f0[l];
                double *pl = part0 + p0[l] * BC;
                if constexpr (half)
                    k_init_h<HT, BC><<<grid, TH, 0, st>>>(g, srcl[l], (float2 *)r + o, hfield_at<HT>(p, o),
                                                          (float2 *)xlo + o, xhi + o, pl, G1[l]);
                else
                    k_init<T, BC><<<grid, TH, 0, st>>>(g, srcl[l], r + o, p + o, xlo ? xlo + o : nullptr,
                                                       xhi ? xhi + o : nullptr, pl, G1[l]);
                s_init<<<Bl[l], SCAL_THREADS, 0, st>>>(B, BC, G1[l], pl, scal_of(l), sph[l], sqrt(tol2));
                if (shifts)
                    k_shift_init<T, TS, BC><<<dim3(Gs1[l], nch[l]), TH, 0, st>>>(
                        V[l], in[l].spec->n_sup, nshift, Bl[l], ch0[l], in[l].spec->d_supsite,
                        in[l].spec->d_rhs_class, r + o, ps + (size_t)nshift * s0[l], y + s0[l], sc, sph[l]);
                ctx->launches += 2 + (shifts ? 1 : 0);
            }
        }
        // the scalar steps ride on the last block of each RHS tile of launches A and B
        const Fuse f1{count, sc, spd, B, 0.0, 0.0, 0.0};
        const Fuse f2{count, sc, spd, B, tol2, delta2, theta2};
        int gyp;
        const Lats Lyp = lats_yp(&gyp);
        const dim3 gridyp(gyp, nchunk);
        const int *rhs_class = in[0].spec->d_rhs_class;
        // two columns per thread for even tiles (SMPQ_HALF_SOLVE_NR=1: one)
#ifndef SMPQ_HALF_SOLVE_NR
#define SMPQ_HALF_SOLVE_NR 2
#endif
        constexpr bool h2cols = SMPQ_HALF_SOLVE_NR == 2 && BC % 2 == 0;
        typedef TileMap<BC, h2cols ? 2 : 1> TMH;
        auto iteration_half = [&](int k) {
            if constexpr (half) {
                const HF<HT> hp = hfield<HT>(p), ht = hfield<HT>(t);
                constexpr int THH = TMH::THREADS;
                int gx;
                const Lats Ld = lats_dw<T, HT>(TMH::SPB, tpb, &gx);
                const dim3 gridh(gx, nchunk);
                auto launch = [&](auto m) {
                    constexpr bool M = decltype(m)::value;
                    if (prof) cudaEventRecord(ctx->prof_ev[4 * k], st);
                    if constexpr (h2cols)
                        k_apply_a_h2<HT, BC, M><<<gridh, THH, 0, st>>>(Ld, hp, ht, (float)kappa, part0, part1, tpb, f1);
                    else
                        k_apply_a_h<HT, BC, M><<<gridh, THH, 0, st>>>(Ld, hp, ht, (float)kappa, part0, part1, tpb, f1);
                    if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 1], st);
                    if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 2], st);
                    if constexpr (h2cols)
                        k_apply_b_h2<HT, BC, M><<<gridh, THH, 0, st>>>(Ld, ht, hp, (float2 *)r, sc.alpha, (float)kappa,
                                                                       part2, tpb, f2);
                    else
                        k_apply_b_h<HT, BC, M><<<gridh, THH, 0, st>>>(Ld, ht, hp, (float2 *)r, sc.alpha, (float)kappa,
                                                                      part2, tpb, f2);
                    if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 3], st);
                    k_yp_h<HT, BC, M><<<gridyp, TH, 0, st>>>(Lyp, nshift, B, rhs_class, (const float2 *)r,
                                                             (float2 *)ps, y, sc, spd, hp, (float2 *)xlo);
                };
                if (multi) launch(std::true_type());
                else launch(std::false_type());
            }
        };
        auto iteration = [&](int k) {
            if constexpr (half) {
                iteration_half(k);
                return;
            }
            // the D_W pair with NR columns per thread, then launch YP
            auto launch = [&](auto nr_c, auto m) {
                constexpr int NR = decltype(nr_c)::value;
                constexpr bool M = decltype(m)::value;
                if constexpr (can_stage && NR == 1) {
                    if (staged) {
                        int gx;
                        const Lats Ld = lats_dw<T>(TileMap<BC>::SPB, tpb, &gx);
                        const dim3 gridn(gx, nchunk);
                        const size_t smem = stage::Dims<BC, stage::NSTAGE>::SMEM;
                        if (prof) cudaEventRecord(ctx->prof_ev[4 * k], st);
                        k_apply_a_st<BC, M><<<gridn, TH, smem, st>>>(Ld, p, t, kd, part0, part1, tpb, f1,
                                                                      sc.flags + 4);
                        if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 1], st);
                        if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 2], st);
                        k_apply_b_st<BC, M><<<gridn, TH, smem, st>>>(Ld, t, p, r, sc.alpha, kd, part2, tpb, f2,
                                                                      sc.flags + 4);
                        if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 3], st);
                        k_yp<T, TS, BC, M><<<gridyp, TH, 0, st>>>(Lyp, nshift, B, rhs_class, r, ps, y, sc, spd, p,
                                                                  xacc, xlo);
                        return;
                    }
                }
                if constexpr (can_stage_df && NR == 1) {
                    if (staged_df) {
                        int gx;
                        const Lats Ld = lats_dw<T>(TileMap<BC>::SPB, tpb, &gx);
                        const dim3 gridn(gx, nchunk);
                        const size_t smem = stage::DimsDF<BC, stage::NSTAGE_DF>::SMEM;
                        if (prof) cudaEventRecord(ctx->prof_ev[4 * k], st);
                        k_apply_a_dfst<BC, M><<<gridn, TH, smem, st>>>(Ld, p, t, kappa, part0, part1, tpb, f1,
                                                                        sc.flags + 4);
                        if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 1], st);
                        if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 2], st);
                        k_apply_b_dfst<BC, M><<<gridn, TH, smem, st>>>(Ld, t, p, r, sc.alpha, kappa, part2, tpb, f2,
                                                                        sc.flags + 4);
                        if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 3], st);
                        k_yp<T, TS, BC, M><<<gridyp, TH, 0, st>>>(Lyp, nshift, B, rhs_class, r, ps, y, sc, spd, p,
                                                                  xacc, xlo);
                        return;
                    }
                }
                if constexpr (NR == 1 || (std::is_same<T, float>::value && BC % 2 == 0 && !M)) {
                    typedef TileMap<BC, NR> TMN;
                    int gx;
                    const Lats Ld = lats_dw<T>(TMN::SPB, tpb, &gx);
                    const dim3 gridn(gx, nchunk);
                    if (prof) cudaEventRecord(ctx->prof_ev[4 * k], st);
                    k_apply_a<T, BC, NR, M><<<gridn, TMN::THREADS, 0, st>>>(Ld, p, t, kd, part0, part1, tpb, f1);
                    if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 1], st);
                    if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 2], st);
                    k_apply_b<T, BC, NR, M><<<gridn, TMN::THREADS, 0, st>>>(Ld, t, p, r, sc.alpha, kd, part2, tpb,
                                                                            f2);
                    if (prof) cudaEventRecord(ctx->prof_ev[4 * k + 3], st);
                    k_yp<T, TS, BC, M><<<gridyp, TH, 0, st>>>(Lyp, nshift, B, rhs_class, r, ps, y, sc, spd, p, xacc, xlo);
                }
            };
            if (multi) launch(std::integral_constant<int, 1>(), std::true_type());
            else if (two_cols) launch(std::integral_constant<int, 2>(), std::false_type());
            else launch(std::integral_constant<int, 1>(), std::false_type());
        };
        // residual replacement, lattice by lattice: x_hi += x_lo, r = b - (A + s0) x_hi in float-float
        auto reliable = [&]() {
            const df64 kdf(ctx->opt.kappa);
            Fuse none{};
            for (int l = 0; l < nl; ++l) {
                const dim3 grid(G1[l], nch[l]);
                const size_t o = f0[l];
                const Geom &g = in[l].ctx->geom;
                const df64c *Udf = (const df64c *)in[l].ctx->Udf.p;
                k_rel_accum<T, BC><<<grid, TH, 0, st>>>(V[l], xhi + o, xlo + o, G1[l]);
                k_apply_a<df64, BC, 1, false><<<grid, TH, 0, st>>>(lats_one<df64>(l), xhi, t64, ctx->opt.kappa, part0,
                                                                   part1, TPB, none);
                k_rel_resid_df<T, BC><<<grid, TH, 0, st>>>(g, Udf, t64 + o, xhi + o, srcl[l], r + o, sph[l].s0, kdf,
                                                           part2 + p0[l] * BC, G1[l]);
                ctx->launches += 3;
            }
            cudaMemsetAsync(sc.flags, 0, 2 * sizeof(int), st);
            for (int l = 0; l < nl; ++l) {
                int base = 0;
                for (int i = 1; i < nshift; ++i)
                    if (sph[l].sig[i] < sph[l].sig[base]) base = i;
                s_rel<<<Bl[l], SCAL_THREADS, 0, st>>>(B, BC, G1[l], part2 + p0[l] * BC, scal_of(l), sph[l], tol2, base);
                ctx->launches += 1;
            }
            // A replacement once every shift has converged (replace_mid = false)
            // re-activates at most the base shift, whose true residual can then be
            // many times the iterated one: its CG restarts from p = r (the old
            // direction belongs to the drifted residual history).
            if (!replace_mid && !half) {
                for (int l = 0; l < nl; ++l) {
                    const size_t nfl = (size_t)12 * V[l] * Bl[l];
                    k_restart_p<C><<<(unsigned)((nfl + 255) / 256), 256, 0, st>>>(r + f0[l], p + f0[l], nfl, BC, V[l],
                                                                                   sc.act_rhs + j0[l]);
                    ctx->launches += 1;
                }
            }
        };
        if (fixed > 0) {
            for (int k = 0; k < fixed; ++k) {
                iteration(prof ? k % chk : 0);
                if (prof && k % chk == chk - 1) {
                    cudaStreamSynchronize(st);
                    collect(chk, hi);
                }
            }
            ctx->launches += (long long)fixed * per_iter;
            iters += fixed;
            return SMPQ_OK;
        }
        // (profiling records CUDA events between launches, so it runs without a graph)
        cudaGraphExec_t gexec = nullptr;
        bool graph_ok = false;
        // the phase that ends at the switch residual checks every 2 iterations:
        // its iterations are the expensive ones, and overshoot would waste them
        const int ck = theta2 > 0 ? std::min(chk, 2) : chk;
        if (ctx->opt.use_graphs && !prof) {
            cudaGraph_t graph;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                for (int k = 0; k < ck; ++k) iteration(k);
                if (cudaStreamEndCapture(st, &graph) == cudaSuccess) {
                    if (cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess) graph_ok = true;
                    cudaGraphDestroy(graph);
                }
            }
            cudaGetLastError();
        }
        int status = SMPQ_OK;
        for (;;) {
            if (graph_ok) cudaGraphLaunch(gexec, st);
            else
                for (int k = 0; k < ck; ++k) iteration(k);
            ctx->launches += (long long)ck * per_iter;
            iters += ck;
            cudaMemcpyAsync(hflags, sc.flags, NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st);
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { status = cuda_check(ctx, e, "multishift iteration"); break; }
            collect(ck, hi);
            if (hflags[4]) {
                status = set_err(ctx, SMPQ_ECUDA, "a shared-memory staging wait of the D_W timed out");
                break;
            }
            if (hflags[2]) { status = set_err(ctx, SMPQ_EBREAKDOWN, "CG breakdown: <p,Ap> <= 0 or not finite"); break; }
            bool done = hflags[0] == 0;
            if (rel && (hflags[1] || done)) {
                reliable();
                ++nrel;
                cudaMemcpyAsync(hflags, sc.flags, NFLAGS * sizeof(int), cudaMemcpyDeviceToHost, st);
                e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) { status = cuda_check(ctx, e, "residual replacement"); break; }
                done = hflags[0] == 0;
            }
            if (done) break;
            if (theta2 > 0 && hflags[3] == 0) break; // every rhs below the switch residual
            if (iters >= max_iter) {
                // the largest relative residual reached, for the message
                std::vector<double> hrr(B), hbb(B);
                cudaMemcpy(hrr.data(), sc.rr, B * sizeof(double), cudaMemcpyDeviceToHost);
                cudaMemcpy(hbb.data(), sc.bb, B * sizeof(double), cudaMemcpyDeviceToHost);
                double worst = 0;
                for (int j = 0; j < B; ++j)
                    if (hbb[j] > 0) worst = std::max(worst, std::sqrt(hrr[j] / hbb[j]));
                char msg[160];
                std::snprintf(msg, sizeof msg, "multishift CG reached max_iter (%d iterations, base residual %.3e)",
                              iters, worst);
                status = set_err(ctx, SMPQ_ENOCONV, msg);
                break;
            }
        }
        if (gexec) cudaGraphExecDestroy(gexec);
        return status;
    }

    // a half field's view at element offset o (components o..., norms o / 12...)
    template <typename HT> HF<HT> hfield_at(void *f, size_t o) const {
        HF<HT> h = hfield<HT>(f);
        return HF<HT>{h.v + o, h.n + o / 12};
    }

    bool relpath = false; // FP32 / half / mixed: the last reliable update left |b - (A + s0) x_hi|^2 in sc.rr

    // True residual of the base system from the FP64 solution x64 (FP64 path):
    // t64 = D_W x64, |b - (D_W^dag t64 + s0 x64)|^2 per rhs into rr_out (the
    // residual itself goes to the scratch field rs).
    int true_residual(double2 *t64, double2 *rs, double *rr_out) {
        const int TH = TileMap<BC>::THREADS;
        for (int l = 0; l < nl; ++l) {
            const dim3 grid(G1[l], nch[l]);
            const size_t o = f0[l];
            smpq_ctx *c = in[l].ctx;
            launch_dslash<double>(c->geom, c->U64.p, x64 + o, t64 + o, Bl[l], BC, 0, ctx->opt.kappa, st);
            k_rel_resid<double, BC><<<grid, TH, 0, st>>>(c->geom, (const double2 *)c->U64.p, t64 + o, x64 + o,
                                                         srcl[l], rs + o, sph[l].s0, ctx->opt.kappa,
                                                         part2 + p0[l] * BC, G1[l]);
            s_sum_rhs<<<Bl[l], SCAL_THREADS, 0, st>>>(BC, G1[l], part2 + p0[l] * BC, rr_out + j0[l]);
            ctx->launches += 3;
        }
        return cuda_check(ctx, cudaGetLastError(), "true residual");
    }

    // The base system's true residual in float-float without replacing r:
    // x_hi += x_lo, t = D_W x_hi, |b - (A + s0) x_hi|^2 per rhs into true_rr
    // (rs: scratch for the residual itself).
    int measure_residual_df(df64c *xhi, float2 *xlo, df64c *t64, float2 *rs) {
        const int TH = TileMap<BC>::THREADS;
        const df64 kdf(ctx->opt.kappa);
        Fuse none{};
        for (int l = 0; l < nl; ++l) {
            const dim3 grid(G1[l], nch[l]);
            const size_t o = f0[l];
            const df64c *Udf = (const df64c *)in[l].ctx->Udf.p;
            k_rel_accum<float, BC><<<grid, TH, 0, st>>>(V[l], xhi + o, xlo + o, G1[l]);
            k_apply_a<df64, BC, 1, false><<<grid, TH, 0, st>>>(lats_one<df64>(l), xhi, t64, ctx->opt.kappa, part0, part1, TPB,
                                                               none);
            k_rel_resid_df<float, BC><<<grid, TH, 0, st>>>(in[l].ctx->geom, Udf, t64 + o, xhi + o, srcl[l], rs + o,
                                                           sph[l].s0, kdf, part2 + p0[l] * BC, G1[l]);
            s_sum_rhs<<<Bl[l], SCAL_THREADS, 0, st>>>(BC, G1[l], part2 + p0[l] * BC, true_rr + j0[l]);
            ctx->launches += 4;
        }
        return cuda_check(ctx, cudaGetLastError(), "true residual");
    }

    int finish(int fixed, const double *d_true_rr = nullptr) {
        cudaEventRecord(ctx->ev2, st);
        std::vector<double> hz((size_t)nshift * B), hrr(B), hbb(B);
        std::vector<int> hit(B);
        std::vector<double> htr(d_true_rr ? B : 0);
        if (d_true_rr) cudaMemcpyAsync(htr.data(), d_true_rr, B * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(hz.data(), sc.zeta, hz.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(hrr.data(), sc.rr, B * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(hbb.data(), sc.bb, B * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(hit.data(), sc.iters, B * sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_check(ctx, e, "multishift statistics");
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev1, ctx->ev2);
        for (int l = 0; l < nl; ++l) {
            double worst = 0, tr = 0;
            int maxit = 0;
            for (int j = j0[l]; j < j0[l] + Bl[l]; ++j) {
                if (!(hbb[j] > 0)) continue;
                for (int i = 0; i < nshift; ++i)
                    worst = std::max(worst, std::fabs(hz[(size_t)i * B + j]) * std::sqrt(hrr[j] / hbb[j]));
                maxit = std::max(maxit, hit[j]);
                tr = std::max(tr, std::sqrt((d_true_rr ? htr[j] : hrr[j]) / hbb[j]));
            }
            SolveOut *out = in[l].out;
            out->y = y + s0[l];
            out->iterations = fixed > 0 ? fixed : maxit;
            out->reliable_updates = nrel;
            out->max_resid = worst;
            out->true_resid = (relpath || d_true_rr) ? tr : -1;
            out->solve_ms = ms;
        }
        return cuda_check(ctx, cudaGetLastError(), "multishift launch");
    }

    // FP64 path with the true_residual option: x64 (and t64 for the final
    // check) on the whole lattice, x64 starting at 0
    int alloc_x64() {
        if (!ctx->opt.true_residual || !shifts) return SMPQ_OK;
        std::vector<Buf> &ws = ctx->ws;
        int rc;
        if ((rc = ensure(ctx, ws[W_XHI], nfield * sizeof(double2)))) return rc;
        if ((rc = ensure(ctx, ws[W_T64], nfield * sizeof(double2)))) return rc;
        x64 = (double2 *)ws[W_XHI].p;
        cudaMemsetAsync(x64, 0, nfield * sizeof(double2), st);
        return SMPQ_OK;
    }

    static int run(const std::vector<LatIn> &lats, double tol, int max_iter, double *hist, int hist_len, int fixed) {
        Solve S(lats);
        smpq_ctx *ctx = S.ctx;
        int rc = S.setup(tol, hist, hist_len);
        if (rc) return rc;
        std::vector<Buf> &ws = ctx->ws;
        const size_t nf = S.nfield;
        const bool shifts = S.shifts;
        const int prec = lats[0].spec->prec;
        const int n = S.nshift;
        cudaEventRecord(ctx->ev1, S.st);
        if (prec == SMPQ_FP64) {
            if ((rc = ensure(ctx, ws[W_P], nf * sizeof(double2)))) return rc;
            if ((rc = ensure(ctx, ws[W_T], nf * sizeof(double2)))) return rc;
            if ((rc = ensure(ctx, ws[W_R], nf * sizeof(double2)))) return rc;
            if (shifts) {
                if ((rc = ensure(ctx, ws[W_PS], (size_t)n * S.nsupf * sizeof(double2)))) return rc;
                if ((rc = ensure(ctx, ws[W_Y], S.nsupf * sizeof(double2)))) return rc;
            }
            S.y = shifts ? (double2 *)ws[W_Y].p : nullptr;
            if ((rc = S.alloc_x64())) return rc;
            rc = S.template phase<double, double>((double2 *)ws[W_P].p, (double2 *)ws[W_T].p, (double2 *)ws[W_R].p,
                                                  nullptr, nullptr, nullptr,
                                                  shifts ? (double2 *)ws[W_PS].p : nullptr, true, false, 0.0, fixed,
                                                  max_iter, S.x64);
            if (rc) return rc;
            if (S.x64 && (rc = S.true_residual((double2 *)ws[W_T64].p, (double2 *)ws[W_R].p, S.true_rr))) return rc;
        } else if (prec == SMPQ_MIXED) {
            // true_residual 0: no base solution is kept (the fastest form);
            // 1: x_hi (float-float, phase 1) and x_lo (FP32, phase 2) accumulate
            // the base solution and its true residual is measured at the end;
            // 2: as 1, and the base system is driven to a true residual below
            // tol (see phase 2)
            const int tres = ctx->opt.true_residual;
            // phase 1: float-float (FP64-accurate) vectors and D_W down to the switch residual
            if ((rc = ensure(ctx, ws[W_P], nf * sizeof(df64c)))) return rc;
            if ((rc = ensure(ctx, ws[W_T], nf * sizeof(df64c)))) return rc;
            if ((rc = ensure(ctx, ws[W_R], nf * sizeof(df64c)))) return rc;
            if (tres && (rc = ensure(ctx, ws[W_XHI], nf * sizeof(df64c)))) return rc;
            if (shifts) {
                if ((rc = ensure(ctx, ws[W_PS], (size_t)n * S.nsupf * sizeof(double2)))) return rc;
                if ((rc = ensure(ctx, ws[W_Y], S.nsupf * sizeof(double2)))) return rc;
            }
            S.y = shifts ? (double2 *)ws[W_Y].p : nullptr;
            double2 *ps = shifts ? (double2 *)ws[W_PS].p : nullptr;
            df64c *p = (df64c *)ws[W_P].p, *t = (df64c *)ws[W_T].p, *r = (df64c *)ws[W_R].p;
            df64c *xh = tres ? (df64c *)ws[W_XHI].p : nullptr;
            const double theta = ctx->opt.switch_residual;
            rc = S.template phase<df64, double>(p, t, r, nullptr, xh, nullptr, ps, true, false, theta * theta, 0,
                                                max_iter, xh);
            if (rc) return rc;
            // phase 2: FP32 vectors and D_W from the phase-1 state, without
            // residual replacement: the FP32 rounding of these iterations makes
            // the base residual drift from the true one by about u_32 theta
            // times a growth factor (measured about 64 u_32 theta: 2.7e-8 at
            // theta = 7e-3), and the shifted systems drift alike.  The drift
            // is smooth over the lattice, so its share of Q = sum_x q(x) does
            // not average out: at theta >= 2e-3 |dQ| over 8^3 x 16 reached
            // 0.5-1.4e-9 for some switch points, at 1e-3 it stays below 3e-11.  With true_residual 2 the base system alone is
            // corrected once every shift has converged (one replacement, then
            // its CG restarts from the true residual): its residual meets tol,
            // but the correction no longer cancels against the other shifts'
            // drift.  The shifted directions are FP32 too (ps32_phase2), y
            // stays FP64.
            const size_t nps = shifts ? (size_t)n * S.nsupf : 0;
            const bool ps32 = ps32_phase2 && shifts;
            if ((rc = ensure(ctx, ws[W_XLO], 4 * nf * sizeof(float2) + (ps32 ? nps * sizeof(float2) : 0)))) return rc;
            float2 *p32 = (float2 *)ws[W_XLO].p, *t32 = p32 + nf, *r32 = t32 + nf, *xl32 = tres ? r32 + nf : nullptr,
                   *ps32p = r32 + 2 * nf;
            const unsigned nb = (unsigned)((nf + 255) / 256);
            k_to_fp32<<<nb, 256, 0, S.st>>>(p, p32, nf);
            k_to_fp32<<<nb, 256, 0, S.st>>>(r, r32, nf);
            if (xl32) cudaMemsetAsync(xl32, 0, nf * sizeof(float2), S.st);
            ctx->launches += 2;
            if (ps32) {
                k_d2f<<<(unsigned)((nps + 255) / 256), 256, 0, S.st>>>(ps, ps32p, nps);
                ctx->launches += 1;
            }
            cudaMemcpyAsync(S.hflags, S.sc.flags, sizeof(int), cudaMemcpyDeviceToHost, S.st);
            cudaStreamSynchronize(S.st);
            const bool enforce = tres == 2;
            if (S.hflags[0] > 0 && enforce) S.relpath = true;
            if (S.hflags[0] > 0 && ps32) {
                rc = S.template phase<float, float>(p32, t32, r32, xl32, xh, t, ps32p, false, enforce, 0.0, 0,
                                                    max_iter, nullptr, false);
                if (rc) return rc;
            } else if (S.hflags[0] > 0) {
                rc = S.template phase<float, double>(p32, t32, r32, xl32, xh, t, ps, false, enforce, 0.0, 0, max_iter,
                                                     nullptr, false);
                if (rc) return rc;
            }
            if (tres == 1) { // measure the base system's true residual (x_hi += x_lo, b - (A + s0) x_hi)
                if ((rc = S.measure_residual_df(xh, xl32, t, r32))) return rc;
                return S.finish(0, S.true_rr);
            }
        } else if (prec == SMPQ_FP16N || prec == SMPQ_BF16N) {
            // p and t in the half format, the rest as in the FP32 path
            const size_t hb = (nf * 4 + nf / 12 * 4 + 255) / 256 * 256;
            if ((rc = ensure(ctx, ws[W_P], hb))) return rc;
            if ((rc = ensure(ctx, ws[W_T], hb))) return rc;
            if ((rc = ensure(ctx, ws[W_R], nf * sizeof(float2)))) return rc;
            if ((rc = ensure(ctx, ws[W_XLO], nf * sizeof(float2)))) return rc;
            if ((rc = ensure(ctx, ws[W_XHI], nf * sizeof(df64c)))) return rc;
            if ((rc = ensure(ctx, ws[W_T64], nf * sizeof(df64c)))) return rc;
            if (shifts) {
                if ((rc = ensure(ctx, ws[W_PS], (size_t)n * S.nsupf * sizeof(float2)))) return rc;
                if ((rc = ensure(ctx, ws[W_Y], S.nsupf * sizeof(double2)))) return rc;
            }
            S.y = shifts ? (double2 *)ws[W_Y].p : nullptr;
            float2 *pp = (float2 *)ws[W_P].p, *tt = (float2 *)ws[W_T].p, *rr = (float2 *)ws[W_R].p;
            float2 *xl = (float2 *)ws[W_XLO].p, *ps = shifts ? (float2 *)ws[W_PS].p : nullptr;
            df64c *xh = (df64c *)ws[W_XHI].p, *t64 = (df64c *)ws[W_T64].p;
            S.relpath = true;
            if (prec == SMPQ_BF16N)
                rc = S.template phase<float, float, B16>(pp, tt, rr, xl, xh, t64, ps, true, true, 0.0, fixed, max_iter);
            else
                rc = S.template phase<float, float, H16>(pp, tt, rr, xl, xh, t64, ps, true, true, 0.0, fixed, max_iter);
            if (rc) return rc;
        } else {
            if ((rc = ensure(ctx, ws[W_P], nf * sizeof(float2)))) return rc;
            if ((rc = ensure(ctx, ws[W_T], nf * sizeof(float2)))) return rc;
            if ((rc = ensure(ctx, ws[W_R], nf * sizeof(float2)))) return rc;
            if ((rc = ensure(ctx, ws[W_XLO], nf * sizeof(float2)))) return rc;
            if ((rc = ensure(ctx, ws[W_XHI], nf * sizeof(df64c)))) return rc;
            if ((rc = ensure(ctx, ws[W_T64], nf * sizeof(df64c)))) return rc;
            if (shifts) {
                if ((rc = ensure(ctx, ws[W_PS], (size_t)n * S.nsupf * sizeof(float2)))) return rc;
                if ((rc = ensure(ctx, ws[W_Y], S.nsupf * sizeof(double2)))) return rc;
            }
            S.y = shifts ? (double2 *)ws[W_Y].p : nullptr;
            S.relpath = true;
            rc = S.template phase<float, float>((float2 *)ws[W_P].p, (float2 *)ws[W_T].p, (float2 *)ws[W_R].p,
                                                (float2 *)ws[W_XLO].p, (df64c *)ws[W_XHI].p, (df64c *)ws[W_T64].p,
                                                shifts ? (float2 *)ws[W_PS].p : nullptr, true, true, 0.0, fixed,
                                                max_iter);
            if (rc) return rc;
        }
        return S.finish(fixed, S.x64 ? S.true_rr : nullptr);
    }
};

int dispatch_bc(const std::vector<LatIn> &lats, double tol, int max_iter, double *hist, int hist_len, int fixed) {
    switch (lats[0].spec->BC) {
    case 1: return Solve<1>::run(lats, tol, max_iter, hist, hist_len, fixed);
    case 12: return Solve<12>::run(lats, tol, max_iter, hist, hist_len, fixed);
    case 24: return Solve<24>::run(lats, tol, max_iter, hist, hist_len, fixed);
    case 48: return Solve<48>::run(lats, tol, max_iter, hist, hist_len, fixed);
    default: return set_err(lats[0].ctx, SMPQ_EINVAL, "unsupported rhs tile width");
    }
}

ShiftParams make_shifts(const smpq_ctx *ctx) {
    ShiftParams sp;
    sp.n = (int)ctx->zq.size();
    sp.s0 = *std::min_element(ctx->zq.begin(), ctx->zq.end());
    for (int i = 0; i < sp.n; ++i) {
        sp.sig[i] = ctx->zq[i] - sp.s0;
        sp.c[i] = ctx->zc[i];
    }
    return sp;
}

} // namespace

int multishift_solve(smpq_ctx *ctx, const SolveSpec &spec, SolveOut *out) {
    if (spec.B % spec.BC) return set_err(ctx, SMPQ_EINVAL, "rhs count must be a multiple of the tile width");
    std::vector<LatIn> lats{LatIn{ctx, &spec, spec.shifts ? *spec.shifts : make_shifts(ctx), out}};
    return dispatch_bc(lats, ctx->opt.tol, ctx->opt.max_iter, nullptr, 0, 0);
}

int multishift_solve_batch(smpq_ctx *const *ctxs, const SolveSpec *specs, SolveOut *outs, int n) {
    if (n < 1 || n > MAX_LAT) return set_err(ctxs[0], SMPQ_EINVAL, "a batched solve takes 1 to 4 lattices");
    std::vector<LatIn> lats;
    for (int l = 0; l < n; ++l) {
        if (specs[l].B % specs[l].BC || specs[l].BC != specs[0].BC || specs[l].prec != specs[0].prec)
            return set_err(ctxs[0], SMPQ_EINVAL, "the lattices of a batched solve need one precision and tile width");
        lats.push_back(LatIn{ctxs[l], &specs[l], specs[l].shifts ? *specs[l].shifts : make_shifts(ctxs[l]), &outs[l]});
    }
    return dispatch_bc(lats, ctxs[0]->opt.tol, ctxs[0]->opt.max_iter, nullptr, 0, 0);
}

// ------------------------------------------------------------------ spectrum (Lanczos from CG coefficients)
__global__ void k_random_source(double2 *b, int V, unsigned long long seed) {
    long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)V * 12) return;
    // splitmix64 of (seed, index): a counter-based generator
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    double u1 = ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    unsigned long long w = z * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    w = (w ^ (w >> 30)) * 0xBF58476D1CE4E5B9ull;
    w = (w ^ (w >> 27)) * 0x94D049BB133111EBull;
    w ^= w >> 31;
    double u2 = ((w >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    b[i] = make_double2(u1 - 0.5, u2 - 0.5);
}

int lanczos_extremes(smpq_ctx *ctx, int iters, double *lo, double *hi) {
    std::vector<Buf> &ws = ctx->ws;
    if (ws.size() < W_COUNT) ws.resize(W_COUNT);
    int rc;
    const int V = ctx->V;
    if ((rc = ensure(ctx, ws[W_B64], (size_t)V * 12 * sizeof(double2) + 2 * (size_t)iters * sizeof(double))))
        return rc;
    double2 *b = (double2 *)ws[W_B64].p;
    double *hist = (double *)(b + (size_t)V * 12);
    k_random_source<<<(V * 12 + 255) / 256, 256, 0, ctx->stream>>>(b, V, 0x5eed5eedull);
    cudaMemsetAsync(hist, 0, 2 * (size_t)iters * sizeof(double), ctx->stream);
    ShiftParams sp;
    sp.n = 1;
    sp.s0 = 0;
    sp.sig[0] = 0;
    sp.c[0] = 0;
    SolveSpec spec{};
    spec.B = 1;
    spec.BC = 1;
    spec.prec = SMPQ_FP64;
    spec.n_sup = 0;
    spec.d_src_field = (const double *)b;
    SolveOut out;
    // the counter lives in the scalar block; reset it through a fresh solve
    std::vector<LatIn> lats{LatIn{ctx, &spec, sp, &out}};
    rc = dispatch_bc(lats, 0.0, iters, hist, iters, iters);
    if (rc) return rc;
    std::vector<double> h(2 * (size_t)iters);
    cudaMemcpyAsync(h.data(), hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "lanczos history");
    // CG -> Lanczos: T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1}, T_{k,k+1} = sqrt(beta_k)/alpha_k
    std::vector<double> diag, off;
    for (int k = 0; k < iters; ++k) {
        double a = h[k], bprev = k > 0 ? h[iters + k - 1] : 0.0, aprev = k > 0 ? h[k - 1] : 1.0;
        if (!(a > 0)) break;
        diag.push_back(1.0 / a + (k > 0 ? bprev / aprev : 0.0));
        double bk = h[iters + k];
        if (k + 1 < iters && h[k + 1] > 0) off.push_back(std::sqrt(bk) / a);
    }
    if (diag.size() < 2) return set_err(ctx, SMPQ_EBREAKDOWN, "Lanczos produced fewer than 2 steps");
    off.resize(diag.size() - 1);
    tridiag_extremes(diag, off, lo, hi);
    return SMPQ_OK;
}

// ------------------------------------------------------------------ autotuner support
// Average time (ms) of one t = D_W p plus one r -= alpha (D_W^dag t + s0 p)
// launch (the two D_W launches of an iteration, without their scalar steps)
// for B right-hand sides in tiles of BC, tpb tiles per block and NR columns
// per thread, on scratch fields (their values do not change the work).
// reps launches each, after one untimed pair.
namespace {
template <typename F> float time_launches(smpq_ctx *ctx, int reps, F once) {
    cudaStream_t st = ctx->stream;
    once(); // warm-up
    cudaEventRecord(ctx->ev1, st);
    for (int k = 0; k < reps; ++k) once();
    cudaEventRecord(ctx->ev2, st);
    if (cudaEventSynchronize(ctx->ev2) != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev1, ctx->ev2);
    return ms / reps;
}

// the table of a single-lattice launch over the context's lattice
Lats lats_single(smpq_ctx *ctx, const void *U, int G) {
    Lats L{};
    L.n = 1;
    L.l[0].g = ctx->geom;
    L.l[0].U = U;
    L.l[0].G = G;
    return L;
}

template <typename T, int BC, int NR>
float time_pair(smpq_ctx *ctx, int B, int tpb, int reps, void *buf, double *part, double *alpha) {
    typedef typename cplx_t<T>::type C;
    typedef TileMap<BC, NR> TM;
    const int V = ctx->V, nchunk = B / BC;
    const int GN = ((V + TM::SPB - 1) / TM::SPB + tpb - 1) / tpb;
    const size_t nf = (size_t)B * 12 * V;
    C *p = (C *)buf, *t = p + nf, *r = t + nf;
    const Lats L = lats_single(ctx, Links<T>::get(ctx), GN);
    cudaStream_t st = ctx->stream;
    const dim3 gridn(GN, nchunk);
    Fuse none{}; // timing only: no scalar step
    return time_launches(ctx, reps, [&]() {
        k_apply_a<T, BC, NR, false><<<gridn, TM::THREADS, 0, st>>>(L, p, t, ctx->opt.kappa, part,
                                                                    part + (size_t)nchunk * GN * BC, tpb, none);
        k_apply_b<T, BC, NR, false><<<gridn, TM::THREADS, 0, st>>>(L, t, p, r, alpha, ctx->opt.kappa, part, tpb, none);
    });
}

// the FP32 pair with staged neighbours (one column per thread); -1 if a
// staging wait ran out (*err, zero on entry)
template <int BC>
float time_pair_staged(smpq_ctx *ctx, int B, int tpb, int reps, void *buf, double *part, double *alpha, int *err) {
    typedef TileMap<BC> TM;
    const int V = ctx->V, nchunk = B / BC;
    const int GN = ((V + TM::SPB - 1) / TM::SPB + tpb - 1) / tpb;
    const size_t nf = (size_t)B * 12 * V;
    float2 *p = (float2 *)buf, *t = p + nf, *r = t + nf;
    const Lats L = lats_single(ctx, Links<float>::get(ctx), GN);
    const double kappa = ctx->opt.kappa;
    cudaStream_t st = ctx->stream;
    const dim3 gridn(GN, nchunk);
    const size_t smem = stage::Dims<BC, stage::NSTAGE>::SMEM;
    if (staged_attrs<BC, false>() != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
    }
    Fuse none{};
    const float ms = time_launches(ctx, reps, [&]() {
        k_apply_a_st<BC, false><<<gridn, TM::THREADS, smem, st>>>(L, p, t, kappa, part,
                                                                   part + (size_t)nchunk * GN * BC, tpb, none, err);
        k_apply_b_st<BC, false><<<gridn, TM::THREADS, smem, st>>>(L, t, p, r, alpha, kappa, part, tpb, none, err);
    });
    int h = 0;
    if (ms < 0 || cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || h) {
        cudaGetLastError();
        return -1.f;
    }
    return ms;
}

// the float-float pair with staged neighbours; -1 if a staging wait ran out
template <int BC>
float time_pair_dfstaged(smpq_ctx *ctx, int B, int tpb, int reps, void *buf, double *part, double *alpha, int *err) {
    typedef TileMap<BC> TM;
    const int V = ctx->V, nchunk = B / BC;
    const int GN = ((V + TM::SPB - 1) / TM::SPB + tpb - 1) / tpb;
    const size_t nf = (size_t)B * 12 * V;
    df64c *p = (df64c *)buf, *t = p + nf, *r = t + nf;
    const Lats L = lats_single(ctx, Links<df64>::get(ctx), GN);
    const df64 kappa(ctx->opt.kappa);
    cudaStream_t st = ctx->stream;
    const dim3 gridn(GN, nchunk);
    const size_t smem = stage::DimsDF<BC, stage::NSTAGE_DF>::SMEM;
    if (staged_df_attrs<BC, false>() != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
    }
    Fuse none{};
    const float ms = time_launches(ctx, reps, [&]() {
        k_apply_a_dfst<BC, false><<<gridn, TM::THREADS, smem, st>>>(L, p, t, kappa, part,
                                                                     part + (size_t)nchunk * GN * BC, tpb, none, err);
        k_apply_b_dfst<BC, false><<<gridn, TM::THREADS, smem, st>>>(L, t, p, r, alpha, kappa, part, tpb, none, err);
    });
    int h = 0;
    if (ms < 0 || cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || h) {
        cudaGetLastError();
        return -1.f;
    }
    return ms;
}

// the half-storage pair (two columns per thread, r and x_lo in FP32)
template <typename HT, int BC>
float time_pair_half(smpq_ctx *ctx, int B, int tpb, int reps, void *buf, double *part, double *alpha) {
    typedef TileMap<BC, 2> TM;
    const int V = ctx->V, nchunk = B / BC;
    const int GN = ((V + TM::SPB - 1) / TM::SPB + tpb - 1) / tpb;
    const size_t nf = (size_t)B * 12 * V;
    const size_t hb = (half_field_bytes(V, B) + 255) / 256 * 256;
    typename HT::h2 *pv = (typename HT::h2 *)buf, *tv = (typename HT::h2 *)((char *)buf + hb);
    const HF<HT> hp{pv, (float *)(pv + nf)}, ht{tv, (float *)(tv + nf)};
    float2 *r = (float2 *)((char *)buf + 2 * hb);
    const Lats L = lats_single(ctx, HLinks<HT>::get(ctx), GN);
    const float kappa = (float)ctx->opt.kappa;
    cudaStream_t st = ctx->stream;
    const dim3 gridn(GN, nchunk);
    Fuse none{};
    return time_launches(ctx, reps, [&]() {
        k_apply_a_h2<HT, BC, false><<<gridn, TM::THREADS, 0, st>>>(L, hp, ht, kappa, part,
                                                                    part + (size_t)nchunk * GN * BC, tpb, none);
        k_apply_b_h2<HT, BC, false><<<gridn, TM::THREADS, 0, st>>>(L, ht, hp, r, alpha, kappa, part, tpb, none);
    });
}

template <int BC> float time_kind(smpq_ctx *ctx, int kind, int B, int tpb, int nr, int reps, void *buf, double *part,
                                  double *alpha, int *err) {
    switch (kind) {
    case 0: return time_pair<double, BC, 1>(ctx, B, tpb, reps, buf, part, alpha);
    case 1:
        return nr == 2 ? time_pair<float, BC, 2>(ctx, B, tpb, reps, buf, part, alpha)
                       : time_pair<float, BC, 1>(ctx, B, tpb, reps, buf, part, alpha);
    case 2: return time_pair<df64, BC, 1>(ctx, B, tpb, reps, buf, part, alpha);
    case 3: return time_pair_half<H16, BC>(ctx, B, tpb, reps, buf, part, alpha);
    case 4: return time_pair_half<B16, BC>(ctx, B, tpb, reps, buf, part, alpha);
    case 5: return time_pair_staged<BC>(ctx, B, tpb, reps, buf, part, alpha, err);
    case 6: return time_pair_dfstaged<BC>(ctx, B, tpb, reps, buf, part, alpha, err);
    default: return -1.f;
    }
}
} // namespace

float time_dslash_pair(smpq_ctx *ctx, int kind, int B, int BC, int tpb, int nr, int reps, void *buf, double *part,
                       double *alpha, int *err) {
    if (tpb < 1 || B % BC) return -1.f;
    switch (BC) {
    case 12: return time_kind<12>(ctx, kind, B, tpb, nr, reps, buf, part, alpha, err);
    case 24: return time_kind<24>(ctx, kind, B, tpb, nr, reps, buf, part, alpha, err);
    case 48: return time_kind<48>(ctx, kind, B, tpb, nr, reps, buf, part, alpha, err);
    default: return -1.f;
    }
}
