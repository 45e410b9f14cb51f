// Float-float ("double-single") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
// bits.  The operations are the error-free transformations of Knuth (two-sum)
// and Dekker (two-product, here with a fused multiply-add), as collected by
// Hida, Li and Bailey (QD library, 2001) and Thall (GPU double-float, 2006).
//
// GB300 executes FP32 about 60 times faster than FP64, so the FP64-accurate
// first phase of the mixed solver runs on this type: the bytes moved are those
// of FP64, the arithmetic stays on the FP32 pipes.  No FP64 instruction is
// issued except in the explicit conversions to and from double.
#pragma once
#include <cuda_runtime.h>

struct __align__(8) df64 {
    float hi, lo;
    __host__ __device__ __forceinline__ df64() {}
    __host__ __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ df64(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ __forceinline__ df64(float v) : hi(v), lo(0.f) {}
    __host__ __device__ __forceinline__ df64(double v) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    }
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ void quick_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    float h, l;
    quick_two_sum(s, e, h, l);
    return df64(h, l);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p); // exact error of the product (Dekker, with FMA)
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    float h, l;
    quick_two_sum(p, e, h, l);
    return df64(h, l);
}
// a * b + c with one renormalisation
__device__ __forceinline__ df64 fma_df(df64 a, df64 b, df64 c) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    float s, t;
    two_sum(p, c.hi, s, t);
    t += e + c.lo;
    float h, l;
    quick_two_sum(s, t, h, l);
    return df64(h, l);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }

struct __align__(16) df64c {
    df64 x, y;
};

// complex helpers with the signatures of smpq_internal.cuh
__device__ __forceinline__ df64c cadd(df64c a, df64c b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ df64c csub(df64c a, df64c b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ df64c cmul(df64c a, df64c b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ df64c cfma(df64c a, df64c b, df64c acc) {
    return {fma_df(a.x, b.x, fma_df(-a.y, b.y, acc.x)), fma_df(a.x, b.y, fma_df(a.y, b.x, acc.y))};
}
__device__ __forceinline__ df64c cfmac(df64c a, df64c b, df64c acc) { // acc + conj(a) b
    return {fma_df(a.x, b.x, fma_df(a.y, b.y, acc.x)), fma_df(a.x, b.y, fma_df(-a.y, b.x, acc.y))};
}
// sum_b a[b] * v[b] over three complex terms with one renormalisation per
// component: the high parts of the six real products of each component are
// summed with two-sum, their exact errors (and the low-part cross terms) in a
// single FP32 accumulator; 70 FP32 operations per component against 90 for a
// chain of fma_df.
__device__ __forceinline__ void ff_prod(float ah, float al, float bh, float bl, float &p, float &q) {
    p = ah * bh;
    q = fmaf(ah, bh, -p);
    q = fmaf(ah, bl, fmaf(al, bh, q));
}
__device__ __forceinline__ void ff_acc(float &s, float &e, float ah, float al, float bh, float bl) {
    float p, q, t, u;
    ff_prod(ah, al, bh, bl, p, q);
    two_sum(s, p, t, u);
    s = t;
    e += q + u;
}
__device__ __forceinline__ df64 ff_finish(float s, float e) {
    float h, l;
    two_sum(s, e, h, l);
    return df64(h, l);
}
__device__ __forceinline__ df64c cdot3(const df64c a[3], const df64c v[3]) {
    float sr, er, si, ei;
    ff_prod(a[0].x.hi, a[0].x.lo, v[0].x.hi, v[0].x.lo, sr, er);
    ff_acc(sr, er, -a[0].y.hi, -a[0].y.lo, v[0].y.hi, v[0].y.lo);
    ff_prod(a[0].x.hi, a[0].x.lo, v[0].y.hi, v[0].y.lo, si, ei);
    ff_acc(si, ei, a[0].y.hi, a[0].y.lo, v[0].x.hi, v[0].x.lo);
#pragma unroll
    for (int b = 1; b < 3; ++b) {
        ff_acc(sr, er, a[b].x.hi, a[b].x.lo, v[b].x.hi, v[b].x.lo);
        ff_acc(sr, er, -a[b].y.hi, -a[b].y.lo, v[b].y.hi, v[b].y.lo);
        ff_acc(si, ei, a[b].x.hi, a[b].x.lo, v[b].y.hi, v[b].y.lo);
        ff_acc(si, ei, a[b].y.hi, a[b].y.lo, v[b].x.hi, v[b].x.lo);
    }
    return {ff_finish(sr, er), ff_finish(si, ei)};
}
// The same sum left unnormalised, (s, e) as the pair; for sums that feed an
// accumulator renormalised later (19 FP32 operations fewer per call).
__device__ __forceinline__ df64c cdot3_lazy(const df64c a[3], const df64c v[3]) {
    float sr, er, si, ei;
    ff_prod(a[0].x.hi, a[0].x.lo, v[0].x.hi, v[0].x.lo, sr, er);
    ff_acc(sr, er, -a[0].y.hi, -a[0].y.lo, v[0].y.hi, v[0].y.lo);
    ff_prod(a[0].x.hi, a[0].x.lo, v[0].y.hi, v[0].y.lo, si, ei);
    ff_acc(si, ei, a[0].y.hi, a[0].y.lo, v[0].x.hi, v[0].x.lo);
#pragma unroll
    for (int b = 1; b < 3; ++b) {
        ff_acc(sr, er, a[b].x.hi, a[b].x.lo, v[b].x.hi, v[b].x.lo);
        ff_acc(sr, er, -a[b].y.hi, -a[b].y.lo, v[b].y.hi, v[b].y.lo);
        ff_acc(si, ei, a[b].x.hi, a[b].x.lo, v[b].y.hi, v[b].y.lo);
        ff_acc(si, ei, a[b].y.hi, a[b].y.lo, v[b].x.hi, v[b].x.lo);
    }
    return {df64(sr, er), df64(si, ei)};
}
// The same unnormalised dot product for two right-hand vectors v0, v1 that
// share the matrix row a (the two spin rows of a projected hop), with packed
// two-lane FP32 instructions (sm_100 and later): lane 0 computes a . v0,
// lane 1 a . v1.
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2b(float a) { return make_float2(a, a); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    float2 bb = __fadd2_rn(s, f2neg(a));
    e = __fadd2_rn(__fadd2_rn(a, f2neg(__fadd2_rn(s, f2neg(bb)))), __fadd2_rn(b, f2neg(bb)));
}
__device__ __forceinline__ void ff_prod2(float2 ah, float2 al, float2 bh, float2 bl, float2 &p, float2 &q) {
    p = __fmul2_rn(ah, bh);
    q = __ffma2_rn(ah, bh, f2neg(p));
    q = __ffma2_rn(ah, bl, __ffma2_rn(al, bh, q));
}
__device__ __forceinline__ void ff_acc2(float2 &s, float2 &e, float2 ah, float2 al, float2 bh, float2 bl) {
    float2 p, q, t, u;
    ff_prod2(ah, al, bh, bl, p, q);
    two_sum2(s, p, t, u);
    s = t;
    e = __fadd2_rn(e, __fadd2_rn(q, u));
}
// lanes: 0 -> a . v0, 1 -> a . v1; (sr, er) real part, (si, ei) imaginary part
__device__ __forceinline__ void cdot3x2_pairs(const df64c a[3], const df64c v0[3], const df64c v1[3], float2 &sr,
                                              float2 &er, float2 &si, float2 &ei) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const float2 axh = f2b(a[b].x.hi), axl = f2b(a[b].x.lo), ayh = f2b(a[b].y.hi), ayl = f2b(a[b].y.lo);
        const float2 vxh = make_float2(v0[b].x.hi, v1[b].x.hi), vxl = make_float2(v0[b].x.lo, v1[b].x.lo);
        const float2 vyh = make_float2(v0[b].y.hi, v1[b].y.hi), vyl = make_float2(v0[b].y.lo, v1[b].y.lo);
        if (b == 0) {
            ff_prod2(axh, axl, vxh, vxl, sr, er);
            ff_prod2(axh, axl, vyh, vyl, si, ei);
        } else {
            ff_acc2(sr, er, axh, axl, vxh, vxl);
            ff_acc2(si, ei, axh, axl, vyh, vyl);
        }
        ff_acc2(sr, er, f2neg(ayh), f2neg(ayl), vyh, vyl);
        ff_acc2(si, ei, ayh, ayl, vxh, vxl);
    }
}
// The same dot products with the right-hand vectors already in packed form:
// (vxh[b], vxl[b], vyh[b], vyl[b]) hold component b of v0 in lane 0 and of v1
// in lane 1.
__device__ __forceinline__ void cdot3x2_packed(const df64c a[3], const float2 vxh[3], const float2 vxl[3],
                                               const float2 vyh[3], const float2 vyl[3], float2 &sr, float2 &er,
                                               float2 &si, float2 &ei) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const float2 axh = f2b(a[b].x.hi), axl = f2b(a[b].x.lo), ayh = f2b(a[b].y.hi), ayl = f2b(a[b].y.lo);
        if (b == 0) {
            ff_prod2(axh, axl, vxh[b], vxl[b], sr, er);
            ff_prod2(axh, axl, vyh[b], vyl[b], si, ei);
        } else {
            ff_acc2(sr, er, axh, axl, vxh[b], vxl[b]);
            ff_acc2(si, ei, axh, axl, vyh[b], vyl[b]);
        }
        ff_acc2(sr, er, f2neg(ayh), f2neg(ayl), vyh[b], vyl[b]);
        ff_acc2(si, ei, ayh, ayl, vxh[b], vxl[b]);
    }
}
// Two complex float-float values in packed form (lane 0, lane 1), unnormalised.
struct f2c {
    float2 xh, xl, yh, yl;
};
// a += (s_x * bx, s_y * by) lazily; the sign pairs are +-1 (exact products)
__device__ __forceinline__ void f2c_add_lazy(f2c &a, float2 sx, float2 sy, float2 bxh, float2 bxl, float2 byh,
                                             float2 byl) {
    float2 t, e;
    two_sum2(a.xh, __fmul2_rn(sx, bxh), t, e);
    a.xh = t;
    a.xl = __fadd2_rn(e, __fadd2_rn(a.xl, __fmul2_rn(sx, bxl)));
    two_sum2(a.yh, __fmul2_rn(sy, byh), t, e);
    a.yh = t;
    a.yl = __fadd2_rn(e, __fadd2_rn(a.yl, __fmul2_rn(sy, byl)));
}
// a + b without the final renormalisation: the high parts are added with
// two-sum, the low parts and the rounding error in plain FP32 (8 operations
// instead of 11).  hi + lo stays exact to about 2^-46 relative but lo may
// exceed half an ulp of hi; renorm() restores the canonical pair.
__device__ __forceinline__ df64 add_lazy(df64 a, df64 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return df64(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ df64 renorm(df64 a) {
    float h, l;
    two_sum(a.hi, a.lo, h, l);
    return df64(h, l);
}
__device__ __forceinline__ df64c cadd_lazy(df64c a, df64c b) { return {add_lazy(a.x, b.x), add_lazy(a.y, b.y)}; }
__device__ __forceinline__ df64c crenorm(df64c a) { return {renorm(a.x), renorm(a.y)}; }
__device__ __forceinline__ df64c cmuli(df64c a) { return {-a.y, a.x}; }
__device__ __forceinline__ df64c cneg(df64c a) { return {-a.x, -a.y}; }
__device__ __forceinline__ df64c cscale(df64 s, df64c a) { return {s * a.x, s * a.y}; }
