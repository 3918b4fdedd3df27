// Double-float arithmetic: the mixed form's loop/branch maps, and every step of
// the double-float product (SIE_PREC_DF).
//
// The loop-space product sums triangle and branch voltages around loops and
// subtree currents along the spanning tree; those sums cancel strongly, so the
// values after the FP32 field computation are carried in more than FP32
// precision.  A double-float value is an unevaluated pair hi + lo of FP32
// numbers (about 48 significant bits); sums and products use the error-free
// transformations two-sum (Knuth) and two-product (one FMA), which run on the
// FP32 pipe.  GB300's FP64 rate is a small fraction of its FP32 rate, so this
// keeps FP64's cancellation safety at FP32 cost.  A complex value is a float4
// (re_hi, re_lo, im_hi, im_lo), the size of a complex128.
#pragma once

#include <cuda_runtime.h>
#include <cmath>

namespace sie {

struct DD {
    float hi, lo;
};

// a + b exactly: hi = fl(a + b), lo the rounding error.
__host__ __device__ __forceinline__ DD two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return DD{s, (a - (s - bb)) + (b - bb)};
}

__host__ __device__ __forceinline__ DD dd_add(DD a, DD b) {
    const DD s = two_sum(a.hi, b.hi);
    const float e = s.lo + (a.lo + b.lo);
    const float hi = s.hi + e;
    return DD{hi, e - (hi - s.hi)};
}

__host__ __device__ __forceinline__ DD dd_neg(DD a) { return DD{-a.hi, -a.lo}; }

// a * b for a double-float a and an FP32 b (a.hi * b exactly by one FMA).
__host__ __device__ __forceinline__ DD dd_mul(DD a, float b) {
    const float p = a.hi * b;
    const float e = fmaf(a.hi, b, -p) + a.lo * b;
    const float hi = p + e;
    return DD{hi, e - (hi - p)};
}

__host__ __device__ __forceinline__ DD dd_mul(DD a, DD b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
    const float hi = p + e;
    return DD{hi, e - (hi - p)};
}

__device__ __forceinline__ DD dd_from(double d) {
    const float hi = __double2float_rn(d);
    return DD{hi, __double2float_rn(d - double(hi))};
}

__device__ __forceinline__ float4 cdd(DD re, DD im) { return make_float4(re.hi, re.lo, im.hi, im.lo); }
__device__ __forceinline__ DD cdd_re(float4 v) { return DD{v.x, v.y}; }
__device__ __forceinline__ DD cdd_im(float4 v) { return DD{v.z, v.w}; }

// A double-float scalar with arithmetic operators: the same hi + lo pair, so
// that the generic field kernels (projection, FFT passes, gathers) instantiate
// for the double-float product (SIE_PREC_DF) as they do for float and double.
// Sums use the two-sum above (error about 2^-44 of the operands' magnitude,
// the usual bound of the short double-float sum), products the FMA two-product.
// Trivially default-constructible so that it can live in shared memory.
struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    // rounding of an FP64 value to the nearest double-float (exact for FP32 values)
    __host__ __device__ constexpr explicit df(double d) : hi(float(d)), lo(float(d - double(float(d)))) {}
};
__host__ __device__ __forceinline__ df operator+(df a, df b) {
    const DD s = dd_add(DD{a.hi, a.lo}, DD{b.hi, b.lo});
    return df(s.hi, s.lo);
}
__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + df(-b.hi, -b.lo); }
__host__ __device__ __forceinline__ df operator*(df a, df b) {
    const DD s = dd_mul(DD{a.hi, a.lo}, DD{b.hi, b.lo});
    return df(s.hi, s.lo);
}
// a * b + c in double-float (the product's error-free FMA part inside dd_mul)
__host__ __device__ __forceinline__ df fma(df a, df b, df c) {
    const DD p = dd_mul(DD{a.hi, a.lo}, DD{b.hi, b.lo});
    const DD s = dd_add(p, DD{c.hi, c.lo});
    return df(s.hi, s.lo);
}
__host__ __device__ __forceinline__ double to_f64(df a) { return double(a.hi) + double(a.lo); }
__host__ __device__ __forceinline__ double to_f64(float a) { return double(a); }
__host__ __device__ __forceinline__ double to_f64(double a) { return a; }
// warp shuffles of one scalar (both halves of a double-float)
__device__ __forceinline__ float shfl1(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl1(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ df shfl1(df v, int src) {
    return df(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
__host__ __device__ __forceinline__ df &operator+=(df &a, df b) { return a = a + b; }
__host__ __device__ __forceinline__ df &operator-=(df &a, df b) { return a = a - b; }
__host__ __device__ __forceinline__ df &operator*=(df &a, df b) { return a = a * b; }
__device__ __forceinline__ DD to_dd(df a) { return DD{a.hi, a.lo}; }

// One local voltage of Eq. Zb with every factor in double-float (the
// double-float product): as dd_zb below with the Gram term g in double-float.
__device__ __forceinline__ float4 dd_zb_df(float2 zr, float2 zi, float2 cl, DD gr, DD gi, DD fr, DD fi) {
    const DD Zr{zr.x, zr.y}, Zi{zi.x, zi.y}, Cl{cl.x, cl.y};
    const DD re = dd_add(dd_add(dd_mul(Zr, gr), dd_neg(dd_mul(Zi, gi))), dd_neg(dd_mul(Cl, fi)));
    const DD im = dd_add(dd_add(dd_mul(Zr, gi), dd_mul(Zi, gr)), dd_mul(Cl, fr));
    return make_float4(re.hi, re.lo, im.hi, im.lo);
}

// One local voltage of Eq. Zb from FP32 field values, carried in double-float:
//   Re y = zr gr - zi gi - cl fi,   Im y = zr gi + zi gr + cl fr,
// with (zr, zi) = Z_s and cl = c_L given as (hi, lo) pairs, g the Gram term and
// f the inductive term.
__device__ __forceinline__ float4 dd_zb(float2 zr, float2 zi, float2 cl, float gr, float gi, DD fr, DD fi) {
    const DD Zr{zr.x, zr.y}, Zi{zi.x, zi.y}, Cl{cl.x, cl.y};
    const DD re = dd_add(dd_add(dd_mul(Zr, gr), dd_neg(dd_mul(Zi, gi))), dd_neg(dd_mul(Cl, fi)));
    const DD im = dd_add(dd_add(dd_mul(Zr, gi), dd_mul(Zi, gr)), dd_mul(Cl, fr));
    return cdd(re, im);
}

}  // namespace sie
