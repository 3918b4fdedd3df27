// Learned correction of the preconditioner's branch diagonal.
//
// The preconditioner of Eq. (Precond) is P = A diag(Z_b) A^T with D_e, the
// diagonal of Z_b (Eq. Zb) on branch e.  The learned form uses
// D'_e = D_e (1 + g(f_e)), with f_e six per-branch features at the frequency
// and g a small network trained on targets the method itself produces (the
// per-branch probing scale of Z_b against D over probe currents).  A network
// whose output layer is zero gives g = 0, the plain preconditioner.
//
// Network (FP32): f [6] -> tanh(W1 f + b1) [H] -> tanh(W2 h1 + b2) [H] ->
// g = 0.5 tanh(w3 . h2 + b3), H = 16 or 32.  Parameters, flat:
// [W1 H x 6][b1 H][W2 H x H][b2 H][w3 H][b3 1].  Training: full-batch mean
// squared error against the targets, gradients by the hand-written backward
// kernel (per-CTA shared-memory accumulation, then one global atomic add per
// parameter and CTA), Adam updates on the device.
#include <cmath>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "sie_plan.h"

using namespace sie;

namespace {

constexpr int kF = 6;
constexpr float kScale = 0.5f;
constexpr double kMu0Over4Pi = 1e-7;

struct Layout {
    int H;
    __host__ __device__ constexpr int W1() const { return 0; }
    __host__ __device__ constexpr int b1() const { return H * kF; }
    __host__ __device__ constexpr int W2() const { return b1() + H; }
    __host__ __device__ constexpr int b2() const { return W2() + H * H; }
    __host__ __device__ constexpr int w3() const { return b2() + H; }
    __host__ __device__ constexpr int b3() const { return w3() + H; }
    __host__ __device__ constexpr int n() const { return b3() + 1; }
};

__device__ __forceinline__ float quarter_decades(double x) {
    const double q = 0.25 * log10(x > 1e-300 ? x : 1e-300);
    return float(q < -20.0 ? -20.0 : (q > 20.0 ? 20.0 : q));
}

// Features of branch e from |Z_s| of its conductor, c_L and the diagonal Gram
// and inductive self terms (the same definition as the oracle's).
__device__ __forceinline__ void branch_features(double zs_abs, double cl, double gd, double ld, float f[kF]) {
    const double a = zs_abs * gd, b = cl * ld;
    f[0] = quarter_decades(a);
    f[1] = quarter_decades(b);
    f[2] = quarter_decades((a > 1e-300 ? a : 1e-300) / (b > 1e-300 ? b : 1e-300));
    f[3] = quarter_decades(gd);
    f[4] = quarter_decades(ld);
    f[5] = quarter_decades(cl / kMu0Over4Pi);
}

template <int H>
__device__ __forceinline__ float mlp_eval(const float *__restrict__ P, const float f[kF], float h1[H], float h2[H],
                                          float &th) {
    constexpr Layout L{H};
#pragma unroll
    for (int i = 0; i < H; ++i) {
        float a = P[L.b1() + i];
#pragma unroll
        for (int k = 0; k < kF; ++k) a += P[L.W1() + i * kF + k] * f[k];
        h1[i] = tanhf(a);
    }
    float z = P[L.b3()];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float a = P[L.b2() + j];
#pragma unroll
        for (int i = 0; i < H; ++i) a += P[L.W2() + j * H + i] * h1[i];
        h2[j] = tanhf(a);
        z += P[L.w3() + j] * h2[j];
    }
    th = tanhf(z);
    return kScale * th;
}

template <int H>
__global__ void __launch_bounds__(128) k_mlp_forward(const float *__restrict__ params, const float *__restrict__ feats,
                                                     int64_t n, float *__restrict__ g) {
    constexpr Layout L{H};
    __shared__ float P[L.n()];
    for (int i = threadIdx.x; i < L.n(); i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float f[kF], h1[H], h2[H], th;
#pragma unroll
    for (int k = 0; k < kF; ++k) f[k] = feats[e * kF + k];
    g[e] = mlp_eval<H>(P, f, h1, h2, th);
}

// Gradient of (1/n) sum (g - t)^2 accumulated into grad (zeroed by the caller);
// the loss into *loss.
template <int H>
__global__ void __launch_bounds__(128) k_mlp_backward(const float *__restrict__ params, const float *__restrict__ feats,
                                                      const float *__restrict__ target, int64_t n,
                                                      float *__restrict__ grad, float *__restrict__ loss) {
    constexpr Layout L{H};
    __shared__ float P[L.n()], G[L.n()];
    __shared__ float lsum;
    for (int i = threadIdx.x; i < L.n(); i += blockDim.x) {
        P[i] = params[i];
        G[i] = 0.f;
    }
    if (threadIdx.x == 0) lsum = 0.f;
    __syncthreads();
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < n) {
        float f[kF], h1[H], h2[H], th;
#pragma unroll
        for (int k = 0; k < kF; ++k) f[k] = feats[e * kF + k];
        const float g = mlp_eval<H>(P, f, h1, h2, th);
        const float r = g - target[e];
        atomicAdd(&lsum, r * r / float(n));
        const float dz = 2.f * r / float(n) * kScale * (1.f - th * th);
        atomicAdd(&G[L.b3()], dz);
        float dh1[H];
#pragma unroll
        for (int i = 0; i < H; ++i) dh1[i] = 0.f;
#pragma unroll
        for (int j = 0; j < H; ++j) {
            atomicAdd(&G[L.w3() + j], dz * h2[j]);
            const float d2 = dz * P[L.w3() + j] * (1.f - h2[j] * h2[j]);
            atomicAdd(&G[L.b2() + j], d2);
#pragma unroll
            for (int i = 0; i < H; ++i) {
                atomicAdd(&G[L.W2() + j * H + i], d2 * h1[i]);
                dh1[i] += d2 * P[L.W2() + j * H + i];
            }
        }
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const float d1 = dh1[i] * (1.f - h1[i] * h1[i]);
            atomicAdd(&G[L.b1() + i], d1);
#pragma unroll
            for (int k = 0; k < kF; ++k) atomicAdd(&G[L.W1() + i * kF + k], d1 * f[k]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L.n(); i += blockDim.x)
        if (G[i] != 0.f) atomicAdd(&grad[i], G[i]);
    if (threadIdx.x == 0) atomicAdd(loss, lsum);
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mi = 0.9f * m[i] + 0.1f * g[i];
    const float vi = 0.999f * v[i] + 0.001f * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void k_branch_features(const double *__restrict__ zs_abs, double cl, const double *__restrict__ gram_diag,
                                  const double *__restrict__ l_diag, const int32_t *__restrict__ br_cond, int64_t nb,
                                  float *__restrict__ out) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    float f[kF];
    branch_features(zs_abs[br_cond[e]], cl, gram_diag[e], l_diag[e], f);
#pragma unroll
    for (int k = 0; k < kF; ++k) out[e * kF + k] = f[k];
}

// t_e = clip(sum_k Re(conj(D_e a_ke) (Z_b a_k)_e) / sum_k |D_e a_ke|^2 - 1), D_e = Z_s G_ee + j c_L Lt_ee.
__global__ void k_probe_target(const double2 *__restrict__ alpha, const double2 *__restrict__ zb_alpha, int32_t k,
                               const double *__restrict__ zs, double cl, const double *__restrict__ gram_diag,
                               const double *__restrict__ l_diag, const int32_t *__restrict__ br_cond, int64_t nb,
                               double clip, float *__restrict__ t) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    const int c = br_cond[e];
    const double dr = zs[2 * c] * gram_diag[e], di = zs[2 * c + 1] * gram_diag[e] + cl * l_diag[e];
    double num = 0.0, den = 0.0;
    for (int32_t q = 0; q < k; ++q) {
        const double2 a = alpha[int64_t(q) * nb + e], z = zb_alpha[int64_t(q) * nb + e];
        const double xr = dr * a.x - di * a.y, xi = dr * a.y + di * a.x;   // D a
        num += xr * z.x + xi * z.y;                                         // Re(conj(D a) Z_b a)
        den += xr * xr + xi * xi;
    }
    double s = den > 0.0 ? num / den - 1.0 : 0.0;
    s = s < -clip ? -clip : (s > clip ? clip : s);
    t[e] = float(s);
}

// a_e /= 1 + g(f_e) for every (frequency slot, branch): the admittances of D'.
template <int H>
__global__ void __launch_bounds__(128) k_learned_admittance(const float *__restrict__ params,
                                                            const double *__restrict__ diag_gram,
                                                            const double *__restrict__ diag_L,
                                                            const int32_t *__restrict__ br_cond,
                                                            const double *__restrict__ zs_cl, int ncond, int64_t nb,
                                                            int32_t nslots, double2 *__restrict__ a) {
    constexpr Layout L{H};
    __shared__ float P[L.n()];
    for (int i = threadIdx.x; i < L.n(); i += blockDim.x) P[i] = params[i];
    __syncthreads();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nb * nslots) return;
    const int64_t f = i / nb, e = i % nb;
    const double *cf = zs_cl + f * (2 * ncond + 1);
    const int c = br_cond[e];
    float feat[kF], h1[H], h2[H], th;
    branch_features(sqrt(cf[2 * c] * cf[2 * c] + cf[2 * c + 1] * cf[2 * c + 1]), cf[2 * ncond], diag_gram[e], diag_L[e],
                    feat);
    const double s = 1.0 / (1.0 + double(mlp_eval<H>(P, feat, h1, h2, th)));
    a[i] = make_double2(a[i].x * s, a[i].y * s);
}

// ---- the width-128 network with FP16 parameters (FP32 arithmetic)
//
// f [6] -> tanh [128] -> tanh [128] -> g = 0.5 tanh(.), every parameter held as
// FP16 (the rounding of FP32 master weights that Adam updates) and converted to
// FP32 for the arithmetic.  A CTA of 128 threads takes tiles of 32 samples:
// thread j computes hidden unit j of every sample of the tile, so the 128 x 128
// layer is a loop of 128 x 32 FMAs per thread over the tile's first-layer
// activations (shared-memory broadcasts) and the FP16 weight column of unit j.
constexpr int kW = 128, kS = 32;

struct alignas(16) Net128 {   // shared-memory copy of the parameters
    float W1[kW * kF], b1[kW], b2[kW], w3[kW], b3;
    __half W2T[kW * kW];   // W2T[i * 128 + j] = W2[j][i]
};

__device__ void load_net128(const __half *__restrict__ p16, Net128 &N, __half *W2 /* [j][i] or null */) {
    constexpr Layout L{kW};
    for (int i = threadIdx.x; i < kW * kF; i += blockDim.x) N.W1[i] = __half2float(p16[L.W1() + i]);
    for (int i = threadIdx.x; i < kW; i += blockDim.x) {
        N.b1[i] = __half2float(p16[L.b1() + i]);
        N.b2[i] = __half2float(p16[L.b2() + i]);
        N.w3[i] = __half2float(p16[L.w3() + i]);
    }
    for (int t = threadIdx.x; t < kW * kW; t += blockDim.x) {
        const int j = t / kW, i = t % kW;   // W2[j][i]
        const __half w = p16[L.W2() + t];
        N.W2T[i * kW + j] = w;
        if (W2) W2[t] = w;
    }
    if (threadIdx.x == 0) N.b3 = __half2float(p16[L.b3()]);
}

// Forward pass of one tile (ft [kS][6] features, ns valid samples): h1, h2
// [kS][128] and th[s] = tanh(z_s); returns through g[s] (s < ns).  Threads:
// 128 (one hidden unit each).
__device__ void fwd_tile128(const Net128 &N, const float *ft, float *h1, float *h2, float *zred, float *th, int ns) {
    const int j = threadIdx.x;
    for (int s = 0; s < kS; ++s) {
        float a = N.b1[j];
#pragma unroll
        for (int k = 0; k < kF; ++k) a += N.W1[j * kF + k] * ft[s * kF + k];
        h1[s * kW + j] = s < ns ? tanhf(a) : 0.f;
    }
    __syncthreads();
    float acc[kS];
#pragma unroll
    for (int s = 0; s < kS; ++s) acc[s] = N.b2[j];
    for (int i = 0; i < kW; i += 4) {
        const float w0 = __half2float(N.W2T[(i + 0) * kW + j]), w1 = __half2float(N.W2T[(i + 1) * kW + j]),
                    w2 = __half2float(N.W2T[(i + 2) * kW + j]), w3 = __half2float(N.W2T[(i + 3) * kW + j]);
#pragma unroll
        for (int s = 0; s < kS; ++s) {
            const float4 h = *reinterpret_cast<const float4 *>(h1 + s * kW + i);
            acc[s] += w0 * h.x + w1 * h.y + w2 * h.z + w3 * h.w;
        }
    }
    const int lane = j & 31, wp = j >> 5;
#pragma unroll
    for (int s = 0; s < kS; ++s) {
        const float h = tanhf(acc[s]);
        h2[s * kW + j] = h;
        float z = N.w3[j] * h;
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        if (lane == 0) zred[wp * kS + s] = z;
    }
    __syncthreads();
    if (j < kS) th[j] = tanhf(N.b3 + zred[j] + zred[kS + j] + zred[2 * kS + j] + zred[3 * kS + j]);
    __syncthreads();
}

__global__ void __launch_bounds__(kW) k_mlp128_forward(const __half *__restrict__ p16, const float *__restrict__ feats,
                                                       int64_t n, float *__restrict__ g) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Net128 &N = *reinterpret_cast<Net128 *>(smraw);
    float *h1 = reinterpret_cast<float *>(smraw + sizeof(Net128));
    float *h2 = h1 + kS * kW, *ft = h2 + kS * kW, *zred = ft + kS * kF, *th = zred + 4 * kS;
    load_net128(p16, N, nullptr);
    for (int64_t t0 = int64_t(blockIdx.x) * kS; t0 < n; t0 += int64_t(gridDim.x) * kS) {
        const int ns = int(n - t0 < kS ? n - t0 : kS);
        __syncthreads();
        for (int q = threadIdx.x; q < kS * kF; q += blockDim.x) ft[q] = q / kF < ns ? feats[t0 * kF + q] : 0.f;
        __syncthreads();
        fwd_tile128(N, ft, h1, h2, zred, th, ns);
        if (threadIdx.x < ns) g[t0 + threadIdx.x] = kScale * th[threadIdx.x];
    }
}

// Gradient of (1/n) sum (g - t)^2 over the CTA's tiles into part[blockIdx.x]
// [param count] and the loss into lpart[blockIdx.x]; accumulators in shared
// memory (gW2 transposed: thread j owns column j).
__global__ void __launch_bounds__(kW) k_mlp128_backward(const __half *__restrict__ p16, const float *__restrict__ feats,
                                                        const float *__restrict__ target, int64_t n,
                                                        float *__restrict__ part, float *__restrict__ lpart) {
    constexpr Layout L{kW};
    extern __shared__ __align__(16) unsigned char smraw[];
    Net128 &N = *reinterpret_cast<Net128 *>(smraw);
    __half *W2 = reinterpret_cast<__half *>(smraw + sizeof(Net128));      // [j][i]
    float *h1 = reinterpret_cast<float *>(W2 + kW * kW);
    float *h2 = h1 + kS * kW, *ft = h2 + kS * kW, *zred = ft + kS * kF, *th = zred + 4 * kS, *dz = th + kS;
    float *gW2T = dz + kS, *gW1 = gW2T + kW * kW, *gb1 = gW1 + kW * kF, *gb2 = gb1 + kW, *gw3 = gb2 + kW;
    float *gsc = gw3 + kW;   // [0] gb3, [1] loss
    load_net128(p16, N, W2);
    const int j = threadIdx.x;
    for (int i = 0; i < kW; ++i) gW2T[i * kW + j] = 0.f;
    for (int k = 0; k < kF; ++k) gW1[j * kF + k] = 0.f;
    gb1[j] = gb2[j] = gw3[j] = 0.f;
    if (j < 2) gsc[j] = 0.f;
    for (int64_t t0 = int64_t(blockIdx.x) * kS; t0 < n; t0 += int64_t(gridDim.x) * kS) {
        const int ns = int(n - t0 < kS ? n - t0 : kS);
        __syncthreads();
        for (int q = j; q < kS * kF; q += blockDim.x) ft[q] = q / kF < ns ? feats[t0 * kF + q] : 0.f;
        __syncthreads();
        fwd_tile128(N, ft, h1, h2, zred, th, ns);
        if (j < kS) {
            float d = 0.f;
            if (j < ns) {
                const float r = kScale * th[j] - target[t0 + j];
                atomicAdd(&gsc[1], r * r / float(n));
                d = 2.f * r / float(n) * kScale * (1.f - th[j] * th[j]);
                atomicAdd(&gsc[0], d);
            }
            dz[j] = d;
        }
        __syncthreads();
        // output layer and the second hidden layer (thread j: unit j)
        float d2[kS];
        float sw = 0.f, sb = 0.f;
#pragma unroll
        for (int s = 0; s < kS; ++s) {
            const float h = h2[s * kW + j];
            sw += dz[s] * h;
            d2[s] = dz[s] * N.w3[j] * (1.f - h * h);
            sb += d2[s];
        }
        gw3[j] += sw;
        gb2[j] += sb;
        for (int i = 0; i < kW; i += 4) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
            for (int s = 0; s < kS; ++s) {
                const float4 h = *reinterpret_cast<const float4 *>(h1 + s * kW + i);
                a0 += d2[s] * h.x;
                a1 += d2[s] * h.y;
                a2 += d2[s] * h.z;
                a3 += d2[s] * h.w;
            }
            gW2T[(i + 0) * kW + j] += a0;
            gW2T[(i + 1) * kW + j] += a1;
            gW2T[(i + 2) * kW + j] += a2;
            gW2T[(i + 3) * kW + j] += a3;
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < kS; ++s) h2[s * kW + j] = d2[s];   // h2 now holds d2[s][j]
        __syncthreads();
        // first hidden layer (thread i = j: unit i): d1[s] = (sum_j W2[j][i] d2[s][j]) (1 - h1^2)
        const int i = j;
        float d1[kS];
#pragma unroll
        for (int s = 0; s < kS; ++s) d1[s] = 0.f;
        for (int jj = 0; jj < kW; jj += 4) {
            const float w0 = __half2float(W2[(jj + 0) * kW + i]), w1 = __half2float(W2[(jj + 1) * kW + i]),
                        w2 = __half2float(W2[(jj + 2) * kW + i]), w3 = __half2float(W2[(jj + 3) * kW + i]);
#pragma unroll
            for (int s = 0; s < kS; ++s) {
                const float4 d = *reinterpret_cast<const float4 *>(h2 + s * kW + jj);
                d1[s] += w0 * d.x + w1 * d.y + w2 * d.z + w3 * d.w;
            }
        }
        float gb = 0.f, gw[kF] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int s = 0; s < kS; ++s) {
            const float h = h1[s * kW + i];
            const float d = d1[s] * (1.f - h * h);
            gb += d;
#pragma unroll
            for (int k = 0; k < kF; ++k) gw[k] += d * ft[s * kF + k];
        }
        gb1[i] += gb;
#pragma unroll
        for (int k = 0; k < kF; ++k) gW1[i * kF + k] += gw[k];
    }
    __syncthreads();
    float *out = part + int64_t(blockIdx.x) * L.n();
    for (int t = j; t < kW * kF; t += blockDim.x) out[L.W1() + t] = gW1[t];
    for (int t = j; t < kW * kW; t += blockDim.x) {
        const int jj = t / kW, ii = t % kW;
        out[L.W2() + t] = gW2T[ii * kW + jj];
    }
    out[L.b1() + j] = gb1[j];
    out[L.b2() + j] = gb2[j];
    out[L.w3() + j] = gw3[j];
    if (j == 0) {
        out[L.b3()] = gsc[0];
        lpart[blockIdx.x] = gsc[1];
    }
}

// grad[p] = sum over the CTAs' partial gradients; loss likewise.
__global__ void k_mlp_reduce(const float *__restrict__ part, const float *__restrict__ lpart, int nblk, int np,
                             float *__restrict__ grad, float *__restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) {
        float a = 0.f;
        for (int b = 0; b < nblk; ++b) a += part[int64_t(b) * np + p];
        grad[p] = a;
    }
    if (p == 0) {
        float l = 0.f;
        for (int b = 0; b < nblk; ++b) l += lpart[b];
        *loss = l;
    }
}

__global__ void k_round_half(const float *__restrict__ p, __half *__restrict__ h, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) h[i] = __float2half_rn(p[i]);
}

// a_e /= 1 + g(f_e) with the width-128 network, tiles of 32 (slot, branch) items.
__global__ void __launch_bounds__(kW) k_learned_admittance128(const __half *__restrict__ p16,
                                                              const double *__restrict__ diag_gram,
                                                              const double *__restrict__ diag_L,
                                                              const int32_t *__restrict__ br_cond,
                                                              const double *__restrict__ zs_cl, int ncond, int64_t nb,
                                                              int32_t nslots, double2 *__restrict__ a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Net128 &N = *reinterpret_cast<Net128 *>(smraw);
    float *h1 = reinterpret_cast<float *>(smraw + sizeof(Net128));
    float *h2 = h1 + kS * kW, *ft = h2 + kS * kW, *zred = ft + kS * kF, *th = zred + 4 * kS;
    load_net128(p16, N, nullptr);
    const int64_t n = nb * int64_t(nslots);
    for (int64_t t0 = int64_t(blockIdx.x) * kS; t0 < n; t0 += int64_t(gridDim.x) * kS) {
        const int ns = int(n - t0 < kS ? n - t0 : kS);
        __syncthreads();
        if (threadIdx.x < kS) {
            float f[kF] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (threadIdx.x < ns) {
                const int64_t i = t0 + threadIdx.x, fs = i / nb, e = i % nb;
                const double *cf = zs_cl + fs * (2 * ncond + 1);
                const int c = br_cond[e];
                branch_features(sqrt(cf[2 * c] * cf[2 * c] + cf[2 * c + 1] * cf[2 * c + 1]), cf[2 * ncond],
                                diag_gram[e], diag_L[e], f);
            }
#pragma unroll
            for (int k = 0; k < kF; ++k) ft[threadIdx.x * kF + k] = f[k];
        }
        __syncthreads();
        fwd_tile128(N, ft, h1, h2, zred, th, ns);
        if (threadIdx.x < ns) {
            const int64_t i = t0 + threadIdx.x;
            const double sc = 1.0 / (1.0 + double(kScale * th[threadIdx.x]));
            a[i] = make_double2(a[i].x * sc, a[i].y * sc);
        }
    }
}

constexpr size_t kSmemFwd128 = sizeof(Net128) + sizeof(float) * (2 * kS * kW + kS * kF + 5 * kS);
constexpr size_t kSmemBwd128 = sizeof(Net128) + sizeof(__half) * kW * kW +
                               sizeof(float) * (2 * kS * kW + kS * kF + 6 * kS + kW * kW + kW * kF + 3 * kW + 2);

// splitmix64 for the initial weights
uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

struct sie_mlp {
    int H = 0;
    int device = 0;
    int64_t t = 0;                      // Adam steps taken
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr, *d_loss = nullptr;
    // width 128: the FP16 parameters the network computes with (rounded from d_p),
    // and the backward pass's per-CTA partial gradients and losses
    __half *d_p16 = nullptr;
    float *d_part = nullptr, *d_lpart = nullptr;
    int nblk = 0;
    int n() const { return Layout{H}.n(); }
};

namespace {
int refresh_half(sie_mlp *m, cudaStream_t st) {
    if (!m->d_p16) return SIE_OK;
    k_round_half<<<(m->n() + 255) / 256, 256, 0, st>>>(m->d_p, m->d_p16, m->n());
    SIE_CUDA(cudaGetLastError());
    return SIE_OK;
}
int set_smem128() {
    SIE_CUDA(cudaFuncSetAttribute((const void *)k_mlp128_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(kSmemFwd128)));
    SIE_CUDA(cudaFuncSetAttribute((const void *)k_learned_admittance128,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemFwd128)));
    SIE_CUDA(cudaFuncSetAttribute((const void *)k_mlp128_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(kSmemBwd128)));
    return SIE_OK;
}
}  // namespace

namespace sie {
// Scale the admittances a [nslots][nb] by 1 / (1 + g) with the plan's learned network.
int learned_admittance(pfft_plan *p, const double *d_zs_cl, int32_t nslots, double2 *a, cudaStream_t st) {
    const sie_mlp *m = p->learned;
    if (!m) return SIE_OK;
    const int64_t n = p->nb * int64_t(nslots);
    const unsigned grid = unsigned((n + 127) / 128);
    if (m->H == kW) {
        int rc = set_smem128();
        if (rc) return rc;
        const int64_t tiles = (n + kS - 1) / kS;
        k_learned_admittance128<<<unsigned(std::min<int64_t>(tiles, 4096)), kW, kSmemFwd128, st>>>(
            m->d_p16, p->d_diag_gram, p->d_diag_L, p->d_br_cond, d_zs_cl, p->ncond, p->nb, nslots, a);
    } else if (m->H == 16)
        k_learned_admittance<16><<<grid, 128, 0, st>>>(m->d_p, p->d_diag_gram, p->d_diag_L, p->d_br_cond, d_zs_cl,
                                                       p->ncond, p->nb, nslots, a);
    else
        k_learned_admittance<32><<<grid, 128, 0, st>>>(m->d_p, p->d_diag_gram, p->d_diag_L, p->d_br_cond, d_zs_cl,
                                                       p->ncond, p->nb, nslots, a);
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}
}  // namespace sie

extern "C" int sie_mlp_create(int32_t hidden, uint64_t seed, sie_mlp **out) {
    if (!out) return fail(SIE_ERR_ARG, "sie_mlp_create: out is NULL");
    *out = nullptr;
    if (hidden != 16 && hidden != 32 && hidden != kW)
        return fail(SIE_ERR_ARG, "sie_mlp_create: hidden width must be 16, 32 or 128");
    sie_mlp *m = new (std::nothrow) sie_mlp;
    if (!m) return fail(SIE_ERR_OOM, "sie_mlp_create: out of host memory");
    m->H = hidden;
    cudaGetDevice(&m->device);
    const Layout L{hidden};
    std::vector<float> p(L.n(), 0.f);
    const double a1 = std::sqrt(6.0 / (kF + hidden)), a2 = std::sqrt(6.0 / (2.0 * hidden));
    uint64_t c = seed * 0x100000001b3ull;
    auto u = [&](double a) { return float(a * (2.0 * double(mix64(c++) >> 11) * (1.0 / 9007199254740992.0) - 1.0)); };
    for (int i = 0; i < hidden * kF; ++i) p[L.W1() + i] = u(a1);
    for (int i = 0; i < hidden * hidden; ++i) p[L.W2() + i] = u(a2);
    const size_t b = size_t(L.n()) * sizeof(float);
    auto bail = [&](cudaError_t e) {
        sie_mlp_destroy(m);
        return fail(SIE_ERR_CUDA, std::string("sie_mlp_create: ") + cudaGetErrorString(e));
    };
    cudaError_t e;
    for (float **d : {&m->d_p, &m->d_g, &m->d_m, &m->d_v})
        if ((e = cudaMalloc(d, b)) != cudaSuccess) return bail(e);
    if ((e = cudaMalloc(&m->d_loss, sizeof(float) * 2)) != cudaSuccess) return bail(e);
    if ((e = cudaMemcpy(m->d_p, p.data(), b, cudaMemcpyHostToDevice)) != cudaSuccess) return bail(e);
    cudaMemset(m->d_m, 0, b);
    cudaMemset(m->d_v, 0, b);
    if (hidden == kW) {
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
        m->nblk = std::max(1, nsm);
        if ((e = cudaMalloc(&m->d_p16, size_t(L.n()) * sizeof(__half))) != cudaSuccess) return bail(e);
        if ((e = cudaMalloc(&m->d_part, size_t(m->nblk) * L.n() * sizeof(float))) != cudaSuccess) return bail(e);
        if ((e = cudaMalloc(&m->d_lpart, size_t(m->nblk) * sizeof(float))) != cudaSuccess) return bail(e);
        if (refresh_half(m, nullptr) || cudaDeviceSynchronize() != cudaSuccess) {
            sie_mlp_destroy(m);
            return fail(SIE_ERR_CUDA, "sie_mlp_create: FP16 copy failed");
        }
    }
    *out = m;
    return SIE_OK;
}

extern "C" void sie_mlp_destroy(sie_mlp *m) {
    if (!m) return;
    for (float *d : {m->d_p, m->d_g, m->d_m, m->d_v, m->d_loss, m->d_part, m->d_lpart})
        if (d) cudaFree(d);
    if (m->d_p16) cudaFree(m->d_p16);
    delete m;
}

extern "C" int64_t sie_mlp_param_count(const sie_mlp *m) { return m ? m->n() : 0; }

extern "C" int sie_mlp_get_params(const sie_mlp *m, float *host, int64_t n) {
    if (!m || !host || n != m->n()) return fail(SIE_ERR_ARG, "sie_mlp_get_params: bad argument");
    SIE_CUDA(cudaMemcpy(host, m->d_p, size_t(n) * sizeof(float), cudaMemcpyDeviceToHost));
    return SIE_OK;
}

extern "C" int sie_mlp_set_params(sie_mlp *m, const float *host, int64_t n) {
    if (!m || !host || n != m->n()) return fail(SIE_ERR_ARG, "sie_mlp_set_params: bad argument");
    SIE_CUDA(cudaMemcpy(m->d_p, host, size_t(n) * sizeof(float), cudaMemcpyHostToDevice));
    SIE_CUDA(cudaMemset(m->d_m, 0, size_t(n) * sizeof(float)));
    SIE_CUDA(cudaMemset(m->d_v, 0, size_t(n) * sizeof(float)));
    m->t = 0;
    int rc = refresh_half(m, nullptr);
    if (rc) return rc;
    SIE_CUDA(cudaDeviceSynchronize());
    return SIE_OK;
}

extern "C" int sie_mlp_forward(const sie_mlp *m, const float *feats, int64_t n, float *g, void *cuda_stream) {
    if (!m || !feats || !g || n < 1) return fail(SIE_ERR_ARG, "sie_mlp_forward: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const unsigned grid = unsigned((n + 127) / 128);
    if (m->H == kW) {
        int rc = set_smem128();
        if (rc) return rc;
        const int64_t tiles = (n + kS - 1) / kS;
        k_mlp128_forward<<<unsigned(std::min<int64_t>(tiles, 4096)), kW, kSmemFwd128, st>>>(m->d_p16, feats, n, g);
    } else if (m->H == 16) {
        k_mlp_forward<16><<<grid, 128, 0, st>>>(m->d_p, feats, n, g);
    } else {
        k_mlp_forward<32><<<grid, 128, 0, st>>>(m->d_p, feats, n, g);
    }
    SIE_CUDA(cudaGetLastError());
    SIE_CUDA(cudaStreamSynchronize(st));
    return SIE_OK;
}

namespace {
int mlp_grad(sie_mlp *m, const float *feats, const float *target, int64_t n, cudaStream_t st) {
    const size_t b = size_t(m->n()) * sizeof(float);
    if (m->H == kW) {   // per-CTA partials in shared memory, then one reduction pass
        int rc = set_smem128();
        if (rc) return rc;
        const int64_t tiles = (n + kS - 1) / kS;
        const int nb = int(std::min<int64_t>(tiles, m->nblk));
        k_mlp128_backward<<<nb, kW, kSmemBwd128, st>>>(m->d_p16, feats, target, n, m->d_part, m->d_lpart);
        SIE_CUDA(cudaGetLastError());
        k_mlp_reduce<<<(m->n() + 255) / 256, 256, 0, st>>>(m->d_part, m->d_lpart, nb, m->n(), m->d_g, m->d_loss);
        SIE_CUDA(cudaGetLastError());
        return SIE_OK;
    }
    SIE_CUDA(cudaMemsetAsync(m->d_g, 0, b, st));
    SIE_CUDA(cudaMemsetAsync(m->d_loss, 0, sizeof(float), st));
    const unsigned grid = unsigned((n + 127) / 128);
    if (m->H == 16) k_mlp_backward<16><<<grid, 128, 0, st>>>(m->d_p, feats, target, n, m->d_g, m->d_loss);
    else k_mlp_backward<32><<<grid, 128, 0, st>>>(m->d_p, feats, target, n, m->d_g, m->d_loss);
    SIE_CUDA(cudaGetLastError());
    return SIE_OK;
}
}  // namespace

extern "C" int sie_mlp_grad(sie_mlp *m, const float *feats, const float *target, int64_t n, float *grad_host,
                            float *loss_host, void *cuda_stream) {
    if (!m || !feats || !target || n < 1) return fail(SIE_ERR_ARG, "sie_mlp_grad: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int rc = mlp_grad(m, feats, target, n, st);
    if (rc) return rc;
    if (grad_host) SIE_CUDA(cudaMemcpyAsync(grad_host, m->d_g, size_t(m->n()) * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (loss_host) SIE_CUDA(cudaMemcpyAsync(loss_host, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    SIE_CUDA(cudaStreamSynchronize(st));
    return SIE_OK;
}

extern "C" int sie_mlp_train(sie_mlp *m, const float *feats, const float *target, int64_t n, int32_t steps, float lr,
                             float *loss_host, void *cuda_stream) {
    if (!m || !feats || !target || n < 1 || steps < 1 || !(lr > 0.f))
        return fail(SIE_ERR_ARG, "sie_mlp_train: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int np = m->n();
    for (int32_t s = 0; s < steps; ++s) {
        int rc = mlp_grad(m, feats, target, n, st);
        if (rc) return rc;
        ++m->t;
        const float c1 = float(1.0 - std::pow(0.9, double(m->t))), c2 = float(1.0 - std::pow(0.999, double(m->t)));
        k_adam<<<(np + 255) / 256, 256, 0, st>>>(m->d_p, m->d_g, m->d_m, m->d_v, np, lr, c1, c2);
        SIE_CUDA(cudaGetLastError());
        if ((rc = refresh_half(m, st))) return rc;
        if (loss_host) SIE_CUDA(cudaMemcpyAsync(loss_host + s, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    SIE_CUDA(cudaStreamSynchronize(st));
    return SIE_OK;
}

extern "C" int pfft_branch_features(pfft_plan *p, double omega, float *feats, void *cuda_stream) {
    if (!p || !feats || !(omega >= 0.0) || !std::isfinite(omega)) return fail(SIE_ERR_ARG, "pfft_branch_features: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<double> za(p->ncond);
    for (int c = 0; c < p->ncond; ++c) za[c] = std::abs(surface_impedance(p, c, omega));
    double *d_za = nullptr;
    SIE_CUDA(cudaMalloc(&d_za, za.size() * sizeof(double)));
    cudaMemcpy(d_za, za.data(), za.size() * sizeof(double), cudaMemcpyHostToDevice);
    k_branch_features<<<unsigned((p->nb + 255) / 256), 256, 0, st>>>(d_za, omega * kMu0Over4Pi, p->d_diag_gram,
                                                                     p->d_diag_L, p->d_br_cond, p->nb, feats);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_za);
    if (e != cudaSuccess) return fail(SIE_ERR_CUDA, std::string("pfft_branch_features: ") + cudaGetErrorString(e));
    return SIE_OK;
}

extern "C" int pfft_branch_probe_target(pfft_plan *p, const void *alpha, int32_t k, double omega, float *target,
                                        void *cuda_stream) {
    if (!p || !alpha || !target || k < 1 || !(omega > 0.0) || !std::isfinite(omega))
        return fail(SIE_ERR_ARG, "pfft_branch_probe_target: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    (void)cudaGetLastError();
    std::vector<double> om(k, omega), zs(2 * p->ncond);
    for (int c = 0; c < p->ncond; ++c) {
        const std::complex<double> z = surface_impedance(p, c, omega);
        zs[2 * c] = z.real();
        zs[2 * c + 1] = z.imag();
    }
    double2 *zb = nullptr;
    double *d_zs = nullptr;
    SIE_CUDA(cudaMalloc(&zb, size_t(k) * p->nb * sizeof(double2)));
    if (cudaMalloc(&d_zs, zs.size() * sizeof(double)) != cudaSuccess) {
        cudaFree(zb);
        return fail(SIE_ERR_OOM, "pfft_branch_probe_target: out of device memory");
    }
    auto done = [&](int rc) {
        cudaFree(zb);
        cudaFree(d_zs);
        return rc;
    };
    cudaMemcpy(d_zs, zs.data(), zs.size() * sizeof(double), cudaMemcpyHostToDevice);
    int rc = matvec_async(p, alpha, zb, k, om.data(), SIE_SPACE_BRANCH, SIE_PREC_FP64, st);
    if (rc) return done(rc);
    k_probe_target<<<unsigned((p->nb + 255) / 256), 256, 0, st>>>(static_cast<const double2 *>(alpha), zb, k, d_zs,
                                                                  omega * kMu0Over4Pi, p->d_diag_gram, p->d_diag_L,
                                                                  p->d_br_cond, p->nb, 0.45, target);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(fail(SIE_ERR_CUDA, std::string("pfft_branch_probe_target: ") + cudaGetErrorString(e)));
    return done(check_device_errors(p));
}

extern "C" int pfft_plan_set_learned(pfft_plan *p, const sie_mlp *m) {
    if (!p) return fail(SIE_ERR_ARG, "pfft_plan_set_learned: NULL plan");
    if (m && m->device != p->device) return fail(SIE_ERR_ARG, "pfft_plan_set_learned: network on another device");
    p->learned = m;
    invalidate_precond_factors(p);
    return SIE_OK;
}
