// Device-side helpers shared by the libsie translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "sie_dd.cuh"
#include "sie_internal.h"

namespace sie {

// complex double-float: 16 bytes like complex128
struct alignas(16) cdf {
    df x, y;
};

template <typename T> struct cpx;
template <> struct cpx<float> { using type = float2; };
template <> struct cpx<double> { using type = double2; };
template <> struct cpx<df> { using type = cdf; };
template <typename T> using C = typename cpx<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T re, T im) { C<T> z; z.x = re; z.y = im; return z; }
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    V z;
    z.x = a.x * b.x - a.y * b.y;
    z.y = a.x * b.y + a.y * b.x;
    return z;
}
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }
// Complex double-float sums and differences leave the pair unnormalised: the
// two-sum of the high parts is exact and its error joins the low parts, with no
// renormalisation (every reader takes hi + lo as the value; products and stores
// normalise).  In the FFT passes a value takes one such add per butterfly stage,
// so its low part stays within a few units of the high part's last place.
__host__ __device__ __forceinline__ df df_qadd(df a, df b) {
    const float s = a.hi + b.hi, bb = s - a.hi;
    return df(s, ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo));
}
template <> __host__ __device__ __forceinline__ cdf cadd<cdf>(cdf a, cdf b) {
    return cdf{df_qadd(a.x, b.x), df_qadd(a.y, b.y)};
}
template <> __host__ __device__ __forceinline__ cdf csub<cdf>(cdf a, cdf b) {
    return cdf{df_qadd(a.x, -b.x), df_qadd(a.y, -b.y)};
}
// multiply by -i (forward) or +i (inverse)
template <typename V> __device__ __forceinline__ V mul_mi(V a, bool inv) {
    V z;
    if (inv) { z.x = -a.y; z.y = a.x; } else { z.x = a.y; z.y = -a.x; }
    return z;
}

// One 3x3 real block of a block-sparse matrix with its column index, packed so
// a warp reads it with a few uniform 16-byte loads: out[a] += sum_b b[3a+b] x[b].
template <typename T> struct Rec;
template <> struct alignas(16) Rec<float> {
    float b[9];
    int32_t col;
    float pad[2];
};
template <> struct alignas(16) Rec<double> {
    double b[9];
    int64_t col;
};
template <> struct alignas(16) Rec<df> {
    df b[9];
    int32_t col;
    int32_t pad;
};
static_assert(sizeof(Rec<float>) == 48 && sizeof(Rec<double>) == 80 && sizeof(Rec<df>) == 80,
              "packed block records");

template <typename T> __device__ __forceinline__ int64_t load_rec(const Rec<T> *__restrict__ r, T (&b)[9]);
template <> __device__ __forceinline__ int64_t load_rec<float>(const Rec<float> *__restrict__ r, float (&b)[9]) {
    const float4 *v = reinterpret_cast<const float4 *>(r);
    const float4 u0 = __ldg(v), u1 = __ldg(v + 1), u2 = __ldg(v + 2);
    b[0] = u0.x; b[1] = u0.y; b[2] = u0.z; b[3] = u0.w;
    b[4] = u1.x; b[5] = u1.y; b[6] = u1.z; b[7] = u1.w;
    b[8] = u2.x;
    return __float_as_int(u2.y);
}
template <> __device__ __forceinline__ int64_t load_rec<double>(const Rec<double> *__restrict__ r, double (&b)[9]) {
    const double2 *v = reinterpret_cast<const double2 *>(r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double2 u = __ldg(v + i);
        b[2 * i] = u.x;
        b[2 * i + 1] = u.y;
    }
    const double2 u = __ldg(v + 4);
    b[8] = u.x;
    return __double_as_longlong(u.y);
}

template <> __device__ __forceinline__ int64_t load_rec<df>(const Rec<df> *__restrict__ r, df (&b)[9]) {
    const float4 *v = reinterpret_cast<const float4 *>(r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 u = __ldg(v + i);
        b[2 * i] = df(u.x, u.y);
        b[2 * i + 1] = df(u.z, u.w);
    }
    const float4 u = __ldg(v + 4);
    b[8] = df(u.x, u.y);
    return __float_as_int(u.z);
}

inline bool cuda_ok(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return true;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return false;
}

}  // namespace sie

#define SIE_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess) {                                                             \
            ::sie::set_error(std::string(#call) + " failed: " + cudaGetErrorString(_e));     \
            return _e == cudaErrorMemoryAllocation ? SIE_ERR_OOM : SIE_ERR_CUDA;             \
        }                                                                                    \
    } while (0)

#define SIE_LAUNCH_CHECK(plan)                                                               \
    do {                                                                                     \
        (plan)->launches++;                                                                  \
        cudaError_t _e = cudaGetLastError();                                                 \
        if (_e != cudaSuccess) {                                                             \
            ::sie::set_error(std::string("kernel launch failed: ") + cudaGetErrorString(_e)); \
            return SIE_ERR_CUDA;                                                             \
        }                                                                                    \
    } while (0)
