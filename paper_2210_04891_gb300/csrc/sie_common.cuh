// Device-side helpers shared by the libsie translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "sie_internal.h"

namespace sie {

template <typename T> struct cpx;
template <> struct cpx<float> { using type = float2; };
template <> struct cpx<double> { using type = double2; };
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
// multiply by -i (forward) or +i (inverse)
template <typename V> __device__ __forceinline__ V mul_mi(V a, bool inv) {
    V z;
    if (inv) { z.x = -a.y; z.y = a.x; } else { z.x = a.y; z.y = -a.x; }
    return z;
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
