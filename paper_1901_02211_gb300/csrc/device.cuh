// Device-side helpers shared by the kernels: complex arithmetic for the three
// iteration types (FP64, FP32, float-float), the lattice geometry and the
// field layout.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "df64.cuh"

// ---------------------------------------------------------------- complex helpers
template <typename T> struct cplx_t;
template <> struct cplx_t<double> { typedef double2 type; };
template <> struct cplx_t<float> { typedef float2 type; };
template <> struct cplx_t<df64> { typedef df64c type; };

// explicit conversion of a real component to double
__host__ __device__ __forceinline__ double to_d(double v) { return v; }
__host__ __device__ __forceinline__ double to_d(float v) { return v; }
__host__ __device__ __forceinline__ double to_d(df64 v) { return (double)v; }

template <typename C> __host__ __device__ __forceinline__ C mkc(double re, double im) {
    C c;
    c.x = re;
    c.y = im;
    return c;
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * b
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
    return acc;
}
// acc + conj(a) * b
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
    return acc;
}
__device__ __forceinline__ float2 cfmac(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
    return acc;
}
// i * a
__device__ __forceinline__ double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
// exact types: lazy addition is plain addition, nothing to renormalise
__device__ __forceinline__ double2 cadd_lazy(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ float2 cadd_lazy(float2 a, float2 b) { return cadd(a, b); }
__device__ __forceinline__ double2 crenorm(double2 a) { return a; }
__device__ __forceinline__ float2 crenorm(float2 a) { return a; }
__device__ __forceinline__ double norm2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double norm2(float2 a) { return (double)a.x * a.x + (double)a.y * a.y; }

// ---------------------------------------------------------------- lattice geometry
struct Geom {
    int n[4];      // nx, ny, nz, nt
    int stride[4]; // 1, nx, nx*ny, nx*ny*nz
    int V;
    float bcf[4];  // boundary factor for hops crossing the boundary in mu
};

// Neighbour of s in direction mu (dir = +1 or -1); *f receives the boundary factor.
__device__ __forceinline__ int neighbour(const Geom &g, int s, int mu, int dir, float *f) {
    int c = (s / g.stride[mu]) % g.n[mu];
    if (dir > 0) {
        if (c == g.n[mu] - 1) {
            *f = g.bcf[mu];
            return s - (g.n[mu] - 1) * g.stride[mu];
        }
        *f = 1.f;
        return s + g.stride[mu];
    }
    if (c == 0) {
        *f = g.bcf[mu];
        return s + (g.n[mu] - 1) * g.stride[mu];
    }
    *f = 1.f;
    return s - g.stride[mu];
}

// ---------------------------------------------------------------- field layout
// A batch of B right-hand sides is stored in RHS tiles of BC columns:
//   element (component c in 0..11 = spin*3 + colour, site s, rhs j)
//   at (((j / BC) * V + s) * 12 + c) * BC + (j % BC),
// i.e. one tile is [site][component][column]: a warp reads consecutive columns
// of one site component, and the 12 components of a site sit at fixed
// offsets (immediates in the load instructions).
// Links: U[(mu * V + s) * 9 + row * 3 + col] (the 9 elements of one link contiguous).
