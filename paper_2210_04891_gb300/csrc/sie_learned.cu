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
    int n() const { return Layout{H}.n(); }
};

namespace sie {
// Scale the admittances a [nslots][nb] by 1 / (1 + g) with the plan's learned network.
int learned_admittance(pfft_plan *p, const double *d_zs_cl, int32_t nslots, double2 *a, cudaStream_t st) {
    const sie_mlp *m = p->learned;
    if (!m) return SIE_OK;
    const int64_t n = p->nb * int64_t(nslots);
    const unsigned grid = unsigned((n + 127) / 128);
    if (m->H == 16)
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
    if (hidden != 16 && hidden != 32) return fail(SIE_ERR_ARG, "sie_mlp_create: hidden width must be 16 or 32");
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
    *out = m;
    return SIE_OK;
}

extern "C" void sie_mlp_destroy(sie_mlp *m) {
    if (!m) return;
    for (float *d : {m->d_p, m->d_g, m->d_m, m->d_v, m->d_loss})
        if (d) cudaFree(d);
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
    return SIE_OK;
}

extern "C" int sie_mlp_forward(const sie_mlp *m, const float *feats, int64_t n, float *g, void *cuda_stream) {
    if (!m || !feats || !g || n < 1) return fail(SIE_ERR_ARG, "sie_mlp_forward: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const unsigned grid = unsigned((n + 127) / 128);
    if (m->H == 16) k_mlp_forward<16><<<grid, 128, 0, st>>>(m->d_p, feats, n, g);
    else k_mlp_forward<32><<<grid, 128, 0, st>>>(m->d_p, feats, n, g);
    SIE_CUDA(cudaGetLastError());
    SIE_CUDA(cudaStreamSynchronize(st));
    return SIE_OK;
}

namespace {
int mlp_grad(sie_mlp *m, const float *feats, const float *target, int64_t n, cudaStream_t st) {
    const size_t b = size_t(m->n()) * sizeof(float);
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
