// pfft_plan_create / destroy / info: the setup of the pre-corrected FFT
// operator of Sec. IV-B of arXiv 2210.04891.
//
// Host (deterministic, FP64, no floating-point contraction): grid spanning the
// mesh box (h_d = extent_d / (N_d - 1)); Radon 7-point sample points per
// triangle with the RWG moments (w_q/2)(r_q - v_k); per point a stencil of the
// O_s nearest nodes per axis with tensor Lagrange weights (Eq. Projection); the
// node -> point gather lists of the projection; the near list (centroid
// distance below r_near or overlapping stencil boxes); Gram blocks.
// Device (FP64): the kernel H(d) = 1/|d o h| on the padded grid and its
// spectrum (Eq. FFTCal, via the same FFT code as the matvec); per near pair
// the direct integral L_direct (closed-form inner integral, outer Gauss rule
// n_touch^2 for pairs sharing a vertex, Radon 7 otherwise) and the grid's own
// contribution (I H B)_pair, L_d = L_direct - (I H B)_pair (Eq. Lb).
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "sie_fft.cuh"
#include "sie_plan.h"

namespace sie {

int plan_alloc(pfft_plan *p, void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + ") failed: " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SIE_ERR_OOM : SIE_ERR_CUDA;
    }
    p->allocations.push_back(*ptr);
    p->device_bytes += bytes;
    return SIE_OK;
}

void plan_free(pfft_plan *p, void *ptr) {
    auto it = std::find(p->allocations.begin(), p->allocations.end(), ptr);
    if (it == p->allocations.end()) return;
    cudaFree(ptr);
    p->allocations.erase(it);
}

template <> const C<double> *twiddle<double>(const pfft_plan *p, int a) { return p->d_tw64[a]; }
template <> const C<float> *twiddle<float>(const pfft_plan *p, int a) { return p->d_tw32[a]; }

}  // namespace sie

using namespace sie;

namespace {

template <typename T>
int upload(pfft_plan *p, T **dst, const std::vector<T> &src) {
    int rc = plan_alloc(p, reinterpret_cast<void **>(dst), src.size() * sizeof(T));
    if (rc) return rc;
    SIE_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SIE_OK;
}

template <typename T>
std::vector<float> to_f32(const std::vector<T> &v) { return std::vector<float>(v.begin(), v.end()); }

// Radon's 7-point degree-5 rule (barycentric points, weights summing to 1).
void radon7(std::vector<double> &bary, std::vector<double> &w) {
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    bary = {1.0 / 3, 1.0 / 3, 1.0 / 3};
    w = {9.0 / 40.0};
    for (int o = 0; o < 2; ++o) {
        double a = o ? a2 : a1, ww = o ? w2 : w1, b = 1.0 - 2.0 * a;
        double pts[3][3] = {{a, a, b}, {a, b, a}, {b, a, a}};
        for (auto &pt : pts) { bary.insert(bary.end(), pt, pt + 3); w.push_back(ww); }
    }
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Conical (collapsed) product rule: (u, v) -> barycentric (1-u-v(1-u), u, v(1-u)).
void collapsed_gauss(int n, std::vector<double> &bary, std::vector<double> &w) {
    std::vector<double> x, wx;
    gauss_legendre(n, x, wx);
    bary.clear();
    w.clear();
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double u = 0.5 * (x[i] + 1.0), v = 0.5 * (x[j] + 1.0);
            double wu = 0.5 * wx[i], wv = 0.5 * wx[j];
            double l1 = u, l2 = v * (1.0 - u);
            bary.push_back(1.0 - l1 - l2);
            bary.push_back(l1);
            bary.push_back(l2);
            w.push_back(wu * wv * (1.0 - u) * 2.0);
        }
}

// ---------------------------------------------------------------- device setup kernels

// K0 = int_S 1/|r-r'| dS', K1 = int_S (rho' - rho)/|r-r'| dS' over triangle v[9]
// (sum over the triangle's edges; see the plan header comment).
__device__ void potentials(const double *r, const double *v, double &K0, double *K1) {
    double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]}, e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    double h = (r[0] - v[0]) * n[0] + (r[1] - v[1]) * n[1] + (r[2] - v[2]) * n[2], ah = fabs(h);
    double rho[3] = {r[0] - h * n[0], r[1] - h * n[1], r[2] - h * n[2]};
    double k0 = 0.0, k1[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        const double *pm = v + 3 * i, *pp = v + 3 * ((i + 1) % 3);
        double L[3] = {pp[0] - pm[0], pp[1] - pm[1], pp[2] - pm[2]};
        double ll = sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
        double lt[3] = {L[0] / ll, L[1] / ll, L[2] / ll};
        double u[3] = {lt[1] * n[2] - lt[2] * n[1], lt[2] * n[0] - lt[0] * n[2], lt[0] * n[1] - lt[1] * n[0]};
        double lp = (pp[0] - rho[0]) * lt[0] + (pp[1] - rho[1]) * lt[1] + (pp[2] - rho[2]) * lt[2];
        double lm = (pm[0] - rho[0]) * lt[0] + (pm[1] - rho[1]) * lt[1] + (pm[2] - rho[2]) * lt[2];
        double P0 = (pm[0] - rho[0]) * u[0] + (pm[1] - rho[1]) * u[1] + (pm[2] - rho[2]) * u[2];
        double R0s = P0 * P0 + h * h;
        double Rp = sqrt((r[0] - pp[0]) * (r[0] - pp[0]) + (r[1] - pp[1]) * (r[1] - pp[1]) + (r[2] - pp[2]) * (r[2] - pp[2]));
        double Rm = sqrt((r[0] - pm[0]) * (r[0] - pm[0]) + (r[1] - pm[1]) * (r[1] - pm[1]) + (r[2] - pm[2]) * (r[2] - pm[2]));
        double f = 0.0;
        if (R0s > 0.0) {
            double num = lp >= 0.0 ? Rp + lp : R0s / (Rp - lp);
            double den = lm >= 0.0 ? Rm + lm : R0s / (Rm - lm);
            f = log(num / den);
        }
        double beta = atan2(P0 * lp, R0s + ah * Rp) - atan2(P0 * lm, R0s + ah * Rm);
        k0 += P0 * f - ah * beta;
        double s = 0.5 * (R0s * f + lp * Rp - lm * Rm);
        k1[0] += s * u[0]; k1[1] += s * u[1]; k1[2] += s * u[2];
    }
    K0 = k0;
    K1[0] = k1[0]; K1[1] = k1[1]; K1[2] = k1[2];
}

// Block[k][l] = int_T (r - v_k)/(2A_T) . int_S (r' - v'_l)/(2A_S) / |r - r'| with T outer.
__device__ void pair_block(const double *vT, double aT, const double *vS, double aS, const double *bary,
                           const double *w, int Q, double *blk) {
    double e1[3] = {vS[3] - vS[0], vS[4] - vS[1], vS[5] - vS[2]}, e2[3] = {vS[6] - vS[0], vS[7] - vS[1], vS[8] - vS[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] /= nn; n[1] /= nn; n[2] /= nn;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < Q; ++q) {
        double r[3], K0, K1[3];
        for (int c = 0; c < 3; ++c) r[c] = bary[3 * q] * vT[c] + bary[3 * q + 1] * vT[3 + c] + bary[3 * q + 2] * vT[6 + c];
        potentials(r, vS, K0, K1);
        double h = (r[0] - vS[0]) * n[0] + (r[1] - vS[1]) * n[1] + (r[2] - vS[2]) * n[2];
        double rho[3] = {r[0] - h * n[0], r[1] - h * n[1], r[2] - h * n[2]};
        for (int k = 0; k < 3; ++k) {
            double o[3] = {r[0] - vT[3 * k], r[1] - vT[3 * k + 1], r[2] - vT[3 * k + 2]};
            for (int l = 0; l < 3; ++l) {
                double in0 = K1[0] + (rho[0] - vS[3 * l]) * K0;
                double in1 = K1[1] + (rho[1] - vS[3 * l + 1]) * K0;
                double in2 = K1[2] + (rho[2] - vS[3 * l + 2]) * K0;
                acc[3 * k + l] += w[q] * (o[0] * in0 + o[1] * in1 + o[2] * in2);
            }
        }
    }
    double s = aT / (4.0 * aT * aS);
    for (int i = 0; i < 9; ++i) blk[i] = acc[i] * s;
}

struct NearArgs {
    const int64_t *ptr;
    const int32_t *col;
    int64_t nt;
    const double *verts;     // [nt][9]
    const double *area;      // [nt]
    const int32_t *tri;      // [nt][3] vertex ids
    const double *r7_bary, *r7_w;
    const double *tg_bary, *tg_w;
    int n_touch_pts;
    // grid part
    const int32_t *start;    // [nt*Q][3]
    const double *lw;        // [nt*Q][3][O]
    const double *mom;       // [nt*Q][3][3]
    const double *Hpad;      // [Mx][My][Mz]
    int Q, O, Mx, My, Mz;
    double *Ldir, *Ld;
};

__device__ int64_t find_row(const int64_t *ptr, int64_t nrows, int64_t e) {
    int64_t lo = 0, hi = nrows;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (ptr[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_near_blocks(NearArgs a, int64_t n_near) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n_near) return;
    int64_t T = find_row(a.ptr, a.nt, e);
    int64_t S = a.col[e];
    int64_t lo = T < S ? T : S, hi = T < S ? S : T;
    bool touch = false;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) touch |= a.tri[3 * lo + i] == a.tri[3 * hi + j];
    double blk[9];
    if (touch)
        pair_block(a.verts + 9 * lo, a.area[lo], a.verts + 9 * hi, a.area[hi], a.tg_bary, a.tg_w, a.n_touch_pts, blk);
    else
        pair_block(a.verts + 9 * lo, a.area[lo], a.verts + 9 * hi, a.area[hi], a.r7_bary, a.r7_w, 7, blk);
    double out[9];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            if (T == S) out[3 * k + l] = 0.5 * (blk[3 * k + l] + blk[3 * l + k]);
            else if (T < S) out[3 * k + l] = blk[3 * k + l];
            else out[3 * k + l] = blk[3 * l + k];
        }
    // grid part: sum_q sum_q' mom_q[k].mom_q'[l] sum_{n in S(q)} sum_{n' in S(q')} L_n H(n - n') L_n'
    // (the same double sum, grouped by the node offset n - n' per axis)
    const int Q = a.Q, O = a.O;
    double g[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < Q; ++q) {
        const int64_t pa = T * Q + q;
        for (int q2 = 0; q2 < Q; ++q2) {
            const int64_t pb = S * Q + q2;
            double cr[3][7];
            int base[3];
            for (int d = 0; d < 3; ++d) {
                const double *la = a.lw + (pa * 3 + d) * O, *lb = a.lw + (pb * 3 + d) * O;
                for (int s = 0; s < 2 * O - 1; ++s) cr[d][s] = 0.0;
                for (int i = 0; i < O; ++i)
                    for (int j = 0; j < O; ++j) cr[d][i - j + O - 1] += la[i] * lb[j];
                base[d] = a.start[3 * pa + d] - a.start[3 * pb + d] - (O - 1);
            }
            double G = 0.0;
            for (int sx = 0; sx < 2 * O - 1; ++sx) {
                int dx = base[0] + sx;
                dx = ((dx % a.Mx) + a.Mx) % a.Mx;
                for (int sy = 0; sy < 2 * O - 1; ++sy) {
                    int dy = base[1] + sy;
                    dy = ((dy % a.My) + a.My) % a.My;
                    const double *row = a.Hpad + (int64_t(dx) * a.My + dy) * a.Mz;
                    double cxy = cr[0][sx] * cr[1][sy];
                    double acc = 0.0;
                    for (int sz = 0; sz < 2 * O - 1; ++sz) {
                        int dz = base[2] + sz;
                        dz = ((dz % a.Mz) + a.Mz) % a.Mz;
                        acc += cr[2][sz] * row[dz];
                    }
                    G += cxy * acc;
                }
            }
            const double *fa = a.mom + 9 * pa, *fb = a.mom + 9 * pb;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l)
                    g[3 * k + l] += (fa[3 * k] * fb[3 * l] + fa[3 * k + 1] * fb[3 * l + 1] + fa[3 * k + 2] * fb[3 * l + 2]) * G;
        }
    }
    for (int i = 0; i < 9; ++i) {
        a.Ldir[9 * e + i] = out[i];
        a.Ld[9 * e + i] = out[i] - g[i];
    }
}

__global__ void k_fill_kernel(double *Hpad, double2 *Hc, int Mx, int My, int Mz, double hx, double hy, double hz,
                              double h0) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t n = int64_t(Mx) * My * Mz;
    if (i >= n) return;
    int iz = int(i % Mz), iy = int((i / Mz) % My), ix = int(i / (int64_t(My) * Mz));
    double v;
    if (ix == Mx / 2 || iy == My / 2 || iz == Mz / 2) {
        v = 0.0;   // offset +-N_d is never used by the aperiodic convolution
    } else {
        int dx = ix < Mx / 2 ? ix : ix - Mx, dy = iy < My / 2 ? iy : iy - My, dz = iz < Mz / 2 ? iz : iz - Mz;
        if (dx == 0 && dy == 0 && dz == 0) {
            v = h0;
        } else {
            double x = __dmul_rn(double(dx), hx), y = __dmul_rn(double(dy), hy), z = __dmul_rn(double(dz), hz);
            double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
            v = __ddiv_rn(1.0, __dsqrt_rn(r2));
        }
    }
    Hpad[i] = v;
    Hc[i] = make_double2(v, 0.0);
}

__global__ void k_extract_H(const double2 *Hc, double *H64, float *H32, int Mx, int My, int Mz, double scale) {
    const int hx = Mx / 2 + 1, hy = My / 2 + 1, hz = Mz / 2 + 1;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(hx) * hy * hz) return;
    int kx = int(i % hx), kz = int((i / hx) % hz), ky = int(i / (int64_t(hx) * hz));
    double v = Hc[(int64_t(kx) * My + ky) * Mz + kz].x * scale;
    H64[i] = v;
    H32[i] = float(v);
}

// The folded spectrum reordered with kx outermost: Hp[kx][ky][kz] = H[ky][kz][kx]
// (all indices folded), so that one x-frequency plane reads a contiguous slice.
__global__ void k_permute_H(const double *H, double *Hp64, float *Hp32, int hx, int hy, int hz) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(hx) * hy * hz) return;
    const int kz = int(i % hz), ky = int((i / hz) % hy), kx = int(i / (int64_t(hy) * hz));
    const double v = H[(int64_t(ky) * hz + kz) * hx + kx];
    Hp64[i] = v;
    Hp32[i] = float(v);
}

// The lossy kernel exp(-jkR)/R, k = (1 - j)/delta, on the padded grid (same
// offsets, wrap and zeroed +-N planes as k_fill_kernel):
// exp(-jkR) = exp(-R/delta) (cos(R/delta) - j sin(R/delta)).
__global__ void k_fill_kernel_lossy(double2 *Hc, int Mx, int My, int Mz, double hx, double hy, double hz, double h0,
                                    double inv_delta) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t n = int64_t(Mx) * My * Mz;
    if (i >= n) return;
    const int iz = int(i % Mz), iy = int((i / Mz) % My), ix = int(i / (int64_t(My) * Mz));
    double2 v = make_double2(0.0, 0.0);
    if (ix != Mx / 2 && iy != My / 2 && iz != Mz / 2) {
        const int dx = ix < Mx / 2 ? ix : ix - Mx, dy = iy < My / 2 ? iy : iy - My, dz = iz < Mz / 2 ? iz : iz - Mz;
        if (dx == 0 && dy == 0 && dz == 0) {
            v = make_double2(h0, 0.0);
        } else {
            const double x = double(dx) * hx, y = double(dy) * hy, z = double(dz) * hz;
            const double r = sqrt(x * x + y * y + z * z);
            const double a = r * inv_delta, m = exp(-a) / r;
            double sn, cs;
            sincos(a, &sn, &cs);
            v = make_double2(m * cs, -m * sn);
        }
    }
    Hc[i] = v;
}

// Complex spectrum folded to one octant with kx outermost, [hx][hy][hz], scaled.
__global__ void k_extract_Hc(const double2 *Hc, double2 *H64, float2 *H32, int Mx, int My, int Mz, double scale) {
    const int hx = Mx / 2 + 1, hy = My / 2 + 1, hz = Mz / 2 + 1;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= int64_t(hx) * hy * hz) return;
    const int kz = int(i % hz), ky = int((i / hz) % hy), kx = int(i / (int64_t(hy) * hz));
    const double2 v = Hc[(int64_t(kx) * My + ky) * Mz + kz];
    H64[i] = make_double2(v.x * scale, v.y * scale);
    H32[i] = make_float2(float(v.x * scale), float(v.y * scale));
}

__global__ void k_branch_diag(const int64_t *ptr, const int32_t *col, const double *Ldir, const int32_t *br_tri,
                              const int8_t *br_local, int64_t nb, double *diagL) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    int32_t t[2] = {br_tri[2 * e], br_tri[2 * e + 1]};
    int k[2] = {br_local[2 * e], br_local[2 * e + 1]};
    double s[2] = {1.0, -1.0};
    double acc = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int64_t end = ptr[t[a] + 1];
            int64_t lo = ptr[t[a]], hi = end;
            while (lo < hi) {   // binary search for column t[b]
                int64_t mid = (lo + hi) / 2;
                if (col[mid] < t[b]) lo = mid + 1; else hi = mid;
            }
            if (lo < end && col[lo] == t[b]) acc += s[a] * s[b] * Ldir[9 * lo + 3 * k[a] + k[b]];
        }
    diagL[e] = acc;
}

// Near blocks and their columns as packed records, FP64 and rounded to FP32.
__global__ void k_pack_near(const int32_t *__restrict__ col, const double *__restrict__ Ld, int64_t n,
                            Rec<double> *__restrict__ r64, Rec<float> *__restrict__ r32) {
    int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n) return;
    Rec<double> a{};
    Rec<float> b{};
    for (int i = 0; i < 9; ++i) {
        a.b[i] = Ld[9 * e + i];
        b.b[i] = float(a.b[i]);
    }
    a.col = col[e];
    b.col = col[e];
    r64[e] = a;
    r32[e] = b;
}

bool is_pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

// Forward 3-D DFT of a full padded complex array hc [Mx][My][Mz] (the kernel
// spectra).  Planes that fit one CTA: (y, z) planes into a temporary, then x
// pencils; otherwise z rows and y pencils in place, then x pencils.  *out is
// hc or the temporary (plan-owned; the caller frees it with plan_free).
int kernel_fft3(pfft_plan *p, double2 *hc, double2 **out, cudaStream_t s) {
    const int64_t nM = int64_t(p->Mx) * p->My * p->Mz;
    double2 *res = hc;
    int rc;
    if (!p->large_plane) {
        const size_t pbytes = size_t(p->My) * p->Mz * sizeof(double2);
        if ((rc = set_smem((const void *)k_fft_plane<double>, pbytes))) return rc;
        if ((rc = plan_alloc(p, (void **)&res, nM * sizeof(double2)))) return rc;
        k_fft_plane<double><<<p->Mx, fft_threads(p->My * p->Mz), pbytes, s>>>(
            hc, int64_t(p->My) * p->Mz, p->My, p->Mz, res, int64_t(p->My) * p->Mz, p->My, p->Mz, p->My, p->Mz,
            p->d_tw64[1], p->d_tw64[2], 0);
        p->launches++;
    } else {
        const int64_t nrows = int64_t(p->Mx) * p->My;
        const int rpc = int(std::min<int64_t>(FFT_E * 256 / p->Mz, nrows));
        const size_t rb = size_t(rpc) * p->Mz * sizeof(double2);
        if ((rc = set_smem((const void *)k_fft_rows<double>, rb))) return rc;
        k_fft_rows<double><<<unsigned(nrows / rpc), 256, rb, s>>>(hc, p->Mz, rpc, p->d_tw64[2]);
        const int kty = std::min(16, p->Mz);
        const size_t yb = size_t(kty) * (p->My + 1) * sizeof(double2);
        if ((rc = set_smem((const void *)k_fft_pencil<double>, yb))) return rc;
        k_fft_pencil<double><<<unsigned(p->Mx * (p->Mz / kty)), fft_threads(kty * p->My), yb, s>>>(
            hc, int64_t(p->My) * p->Mz, p->Mz, p->My, p->My, p->My, p->My, p->Mz, kty, p->d_tw64[1], nullptr);
        p->launches += 2;
    }
    const int KT = 16, ncols = p->My * p->Mz;
    const size_t kb = size_t(KT) * (p->Mx + 1) * sizeof(double2);
    if ((rc = set_smem((const void *)k_fft_pencil<double>, kb))) return rc;
    k_fft_pencil<double><<<ncols / KT, fft_threads(KT * p->Mx), kb, s>>>(res, 0, ncols, p->Mx, p->Mx, p->Mx, p->My,
                                                                       p->Mz, KT, p->d_tw64[0], nullptr);
    p->launches++;
    SIE_CUDA(cudaGetLastError());
    *out = res;
    return SIE_OK;
}

}  // namespace

namespace sie {

// The dynamic shared-memory limit is an attribute of the function on a device,
// shared by every plan and host thread, while the bytes a launch needs can
// differ from plan to plan (band widths, front sizes, plane sizes).  So the
// limit is only ever raised, under a lock: a plan needing less can never lower
// it between another thread's setting and that thread's launch.  It is raised
// for requests below 48 KB too: the default limit is 48 KB less the kernel's
// static shared memory.
int set_smem(const void *fn, size_t bytes) {
    int dev = 0;
    SIE_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> limit;
    std::lock_guard<std::mutex> lock(mu);
    size_t &cur = limit[std::make_pair(fn, dev)];
    if (bytes > cur) {
        SIE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
        cur = bytes;
    }
    return SIE_OK;
}


// FFT convolution of ngrids grids [Nx][Ny][Nz] (in `grid`, overwritten with
// the result) through the buffer `spec` [ngrids][Mx][Ny][Nz]: x pencils
// forward, then per x-frequency plane the zero-padded (y, z) transform, the
// kernel product and the inverse (y, z) transform, then x pencils inverse.
// Only the x-padded grid (2 N_g per grid) goes through device memory.
template <typename T> struct Tables;
template <> struct Tables<double> {
    static const double2 *tf(const pfft_plan *p, int a) { return p->d_tf64[a]; }
    static const double2 *ti(const pfft_plan *p, int a) { return p->d_ti64[a]; }
    static const double *Hp(const pfft_plan *p) { return p->d_Hp64; }
    static const double2 *Hl(const pfft_plan *p) { return p->d_Hl64; }
};
template <> struct Tables<float> {
    static const float2 *tf(const pfft_plan *p, int a) { return p->d_tf32[a]; }
    static const float2 *ti(const pfft_plan *p, int a) { return p->d_ti32[a]; }
    static const float *Hp(const pfft_plan *p) { return p->d_Hp32; }
    static const float2 *Hl(const pfft_plan *p) { return p->d_Hl32; }
};
template <> struct Tables<df> {   // the double-float product: static kernel only
    static const cdf *tf(const pfft_plan *p, int a) { return p->d_tfdf[a]; }
    static const cdf *ti(const pfft_plan *p, int a) { return p->d_tidf[a]; }
    static const df *Hp(const pfft_plan *p) { return p->d_Hpdf; }
};

// Pencils along axis `axis` (0: x, ncols = N_y N_z per grid; 1: y of the large
// plane route, ncols = N_z per (grid, x-frequency)) for `nbatch` batches.
template <typename T, int N1, int N2>
int launch_pencils(pfft_plan *p, const C<T> *in, C<T> *out, int64_t nbatch, int ncols, int axis, bool inverse,
                   cudaStream_t s) {
    using Tb = Tables<T>;
    using Pc = Pencil<N1, N2>;
    const size_t pb = size_t(Pc::KT) * (N1 * N2 + 1) * sizeof(C<T>);
    const int64_t ctas = nbatch * (ncols / Pc::KT);
    if (ncols % Pc::KT || ctas > INT32_MAX) return fail(SIE_ERR_ARG, "pencil FFT: unsupported shape");
    if (!inverse) {
        int rc = set_smem((const void *)k_fft_xf<T, N1, N2>, pb);
        if (rc) return rc;
        k_fft_xf<T, N1, N2><<<unsigned(ctas), Pc::threads, pb, s>>>(in, out, ncols, Tb::tf(p, axis));
    } else {
        int rc = set_smem((const void *)k_fft_xi<T, N1, N2>, pb);
        if (rc) return rc;
        k_fft_xi<T, N1, N2><<<unsigned(ctas), Pc::threads, pb, s>>>(in, out, ncols, Tb::ti(p, axis));
    }
    return SIE_OK;
}

template <typename T, int N1, int N2>
int launch_x(pfft_plan *p, const C<T> *in, C<T> *out, int ngrids, bool inverse, cudaStream_t s) {
    return launch_pencils<T, N1, N2>(p, in, out, ngrids, p->Ny * p->Nz, 0, inverse, s);
}

// z rows of the large plane route: forward, kernel product, inverse, in place.
template <typename T, int N1, int N2, typename HT>
int launch_zconv(pfft_plan *p, C<T> *rows, int64_t nrows, const HT *Hp, const HT *const *Htab, const int32_t *gslot,
                 cudaStream_t s) {
    using Tb = Tables<T>;
    using Z = ZRows<N1, N2>;
    const size_t zb = size_t(Z::RPC) * Z::pitch * sizeof(C<T>);
    if (nrows % Z::RPC || nrows / Z::RPC > INT32_MAX) return fail(SIE_ERR_ARG, "z-row FFT: unsupported shape");
    int rc = set_smem((const void *)k_fft_zconv<T, N1, N2, HT>, zb);
    if (rc) return rc;
    int lgMx = 0, lgMy = 0;
    while ((1 << lgMx) < p->Mx) ++lgMx;
    while ((1 << lgMy) < p->My) ++lgMy;
    k_fft_zconv<T, N1, N2, HT><<<unsigned(nrows / Z::RPC), 256, zb, s>>>(rows, lgMx, lgMy, Hp, Tb::tf(p, 2),
                                                                          Tb::ti(p, 2), Htab, gslot);
    return SIE_OK;
}

// (y, z) convolution of the x-transformed grids when the plane does not fit
// one CTA: y pencils forward into the second half of `spec`, z rows (forward,
// kernel product, inverse), y pencils inverse back into the first half.
template <typename T, typename HT>
int launch_yz_large(pfft_plan *p, C<T> *spec, int32_t ngrids, const HT *Hp, const HT *const *Htab,
                    const int32_t *gslot, cudaStream_t s) {
    const int64_t planes = int64_t(ngrids) * p->Mx;
    C<T> *spec2 = spec + planes * p->Ny * p->Nz;
    int rc;
    SIE_SPLIT_DISPATCH_P(p->My, (rc = launch_pencils<T, N1, N2>(p, spec, spec2, planes, p->Nz, 1, false, s)));
    if (rc) return rc;
    SIE_LAUNCH_CHECK(p);
    SIE_SPLIT_DISPATCH_P(p->Mz, (rc = launch_zconv<T, N1, N2, HT>(p, spec2, planes * p->My, Hp, Htab, gslot, s)));
    if (rc) return rc;
    SIE_LAUNCH_CHECK(p);
    SIE_SPLIT_DISPATCH_P(p->My, (rc = launch_pencils<T, N1, N2>(p, spec2, spec, planes, p->Nz, 1, true, s)));
    if (rc) return rc;
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

template <typename T, typename HT>
int launch_yzc(pfft_plan *p, C<T> *spec, int32_t ngrids, const HT *Hp, cudaStream_t s,
               const HT *const *Htab = nullptr, const int32_t *gslot = nullptr) {
    using Tb = Tables<T>;
    if (p->large_plane) return launch_yz_large<T, HT>(p, spec, ngrids, Hp, Htab, gslot, s);
    if constexpr (sizeof(T) == 4 && sizeof(HT) == sizeof(T)) {   // static kernel in FP32: paired form
        bool done = false;
        const int rc = plane_conv_f32(p, spec, ngrids, s, done);
        if (rc || done) return rc;
    }
    // 512 threads for the FP32 static kernel (64 registers); the complex kernel value needs more
    constexpr int NT = (sizeof(T) == 4 && sizeof(HT) == sizeof(T)) ? 512 : 256;
    const size_t plane_bytes = size_t(p->My + p->Ny) * (p->Mz + 1) * sizeof(C<T>);
    int rc = set_smem((const void *)k_fft_yzc<T, NT, HT>, plane_bytes);
    if (rc) return rc;
    int lgMx = 0;
    while ((1 << lgMx) < p->Mx) ++lgMx;
    k_fft_yzc<T, NT, HT><<<unsigned(ngrids * p->Mx), NT, plane_bytes, s>>>(spec, lgMx, p->My, p->Mz, Hp, Tb::tf(p, 1),
                                                                        Tb::ti(p, 1), Tb::tf(p, 2), Tb::ti(p, 2),
                                                                        Htab, gslot);
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

template <typename T>
int fft_conv_t(pfft_plan *p, C<T> *grid, C<T> *spec, int32_t ngrids, cudaStream_t s, bool lossy,
               const SpecSel *sel) {
    using Tb = Tables<T>;
    int rc;
    {
        StageTimer tm(p, SIE_STAGE_FFT_X_FWD, s);
        SIE_SPLIT_DISPATCH_P(p->Mx, (rc = launch_x<T, N1, N2>(p, grid, spec, ngrids, false, s)));
        if (rc) return rc;
        SIE_LAUNCH_CHECK(p);
    }
    {
        StageTimer tm(p, SIE_STAGE_FFT_YZ, s);
        if constexpr (std::is_same<T, df>::value)
            rc = launch_yzc<T>(p, spec, ngrids, Tb::Hp(p), s);
        else if (sel && sel->tab)   // one lossy spectrum per grid
            rc = launch_yzc<T, C<T>>(p, spec, ngrids, nullptr, s, reinterpret_cast<const C<T> *const *>(sel->tab),
                                     sel->gslot);
        else
            rc = lossy ? launch_yzc<T>(p, spec, ngrids, Tb::Hl(p), s) : launch_yzc<T>(p, spec, ngrids, Tb::Hp(p), s);
        if (rc) return rc;
    }
    StageTimer tm(p, SIE_STAGE_FFT_X_INV, s);
    SIE_SPLIT_DISPATCH_P(p->Mx, (rc = launch_x<T, N1, N2>(p, spec, grid, ngrids, true, s)));
    if (rc) return rc;
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

int fft_conv_n(pfft_plan *p, void *grid, void *spec, int32_t ngrids, int prec, cudaStream_t s, bool lossy,
               const SpecSel *sel) {
    if (prec == SIE_PREC_FP64) return fft_conv_t<double>(p, (double2 *)grid, (double2 *)spec, ngrids, s, lossy, sel);
    if (prec == SIE_PREC_DF) {
        if (lossy || !p->df_ready) return fail(SIE_ERR_ARG, "double-float convolution: static kernel, tables built");
        return fft_conv_t<df>(p, (cdf *)grid, (cdf *)spec, ngrids, s, false, nullptr);
    }
    return fft_conv_t<float>(p, (float2 *)grid, (float2 *)spec, ngrids, s, lossy, sel);
}

int fft_conv(pfft_plan *p, void *grid, void *spec, int32_t nrhs, int prec, cudaStream_t s, const SpecSel *sel) {
    return fft_conv_n(p, grid, spec, 3 * nrhs, prec, s, sel != nullptr, sel);
}

// Reads and clears the plan's device error flags (call after the work that
// may have set them has completed).
int check_device_errors(pfft_plan *p) {
    int flags = 0;
    SIE_CUDA(cudaMemcpy(&flags, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!flags) return SIE_OK;
    SIE_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
    return fail(SIE_ERR_TIMEOUT, "a bounded device-side wait ran out (tensor-core near field); results are invalid");
}

int finish_call(pfft_plan *p, cudaStream_t st) {
    if (!p->h_err) {
        SIE_CUDA(cudaStreamSynchronize(st));
        return check_device_errors(p);
    }
    SIE_CUDA(cudaMemcpyAsync(p->h_err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SIE_CUDA(cudaStreamSynchronize(st));
    if (!*p->h_err) return SIE_OK;
    SIE_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
    *p->h_err = 0;
    return fail(SIE_ERR_TIMEOUT, "a bounded device-side wait ran out (tensor-core near field); results are invalid");
}

}  // namespace sie

extern "C" int pfft_plan_create(const sie_mesh *m, const sie_loops *L, const pfft_params *prm, void *cuda_stream,
                                pfft_plan **out) {
    if (!m || !L || !prm || !out) return fail(SIE_ERR_ARG, "pfft_plan_create: NULL argument");
    *out = nullptr;
    if (L->nt != m->nt) return fail(SIE_ERR_ARG, "pfft_plan_create: loops built for another mesh");
    const int O = prm->order;
    if (O < 2 || O > 4) return fail(SIE_ERR_ARG, "pfft_plan_create: order must be 2..4");
    for (int d = 0; d < 3; ++d)
        if (!is_pow2(prm->grid[d]) || prm->grid[d] < O || prm->grid[d] < 4 || prm->grid[d] > 256)
            return fail(SIE_ERR_ARG, "pfft_plan_create: grid sizes must be powers of two in [max(4, order), 256]");
    // the padded (y, z) plane fits one CTA's shared memory in FP64 (2N_y 2N_z <= 8192 and
    // 3 N_y (2N_z + 1) 16 B <= 200 KiB); otherwise y pencils of N_z columns and z rows
    const int gy = prm->grid[1], gz = prm->grid[2];
    const bool plane_fits = gy <= 128 && gz <= 128 && 3 * gy * (2 * gz + 1) * 16 <= 200 * 1024 &&
                            4 * gy * gz <= FFT_MAX_ELEMS;
    if (!plane_fits && gz % (2 * gy > 256 ? 8 : 16) != 0)
        return fail(SIE_ERR_ARG, "pfft_plan_create: a padded y-z plane larger than one CTA needs N_z >= 16 "
                                 "(N_z >= 8 when N_y = 256)");
    if (prm->n_touch < 1 || prm->n_touch > 64) return fail(SIE_ERR_ARG, "pfft_plan_create: n_touch must be 1..64");
    if (!(prm->near_factor >= 0.0) || !(prm->near_min_diam >= 0.0)) return fail(SIE_ERR_ARG, "pfft_plan_create: negative near radius");
    if (prm->kernel != SIE_KERNEL_STATIC && prm->kernel != SIE_KERNEL_LOSSY)
        return fail(SIE_ERR_ARG, "pfft_plan_create: kernel must be SIE_KERNEL_STATIC or SIE_KERNEL_LOSSY");
    if (prm->kernel == SIE_KERNEL_LOSSY)
        for (int32_t c = 1; c < m->ncond; ++c)
            if (m->sigma[c] != m->sigma[0])
                return fail(SIE_ERR_ARG, "pfft_plan_create: the lossy kernel needs one conductivity for every conductor");

    (void)cudaGetLastError();   // a stale error from earlier work in this thread is not ours
    pfft_plan *p = new (std::nothrow) pfft_plan;
    if (!p) return fail(SIE_ERR_OOM, "pfft_plan_create: out of host memory");
    auto bail = [&](int rc) { pfft_plan_destroy(p); return rc; };
    cudaGetDevice(&p->device);
    p->stream = static_cast<cudaStream_t>(cuda_stream);
    p->params = *prm;
    p->loops = L;
    p->nt = m->nt; p->nb = L->nb; p->nl = L->nl; p->np = L->np; p->nn = L->n_nodes;
    p->ncond = m->ncond;
    p->sigma = m->sigma;
    p->t_eff.assign(p->sigma.size(), 0.0);
    p->O = O;
    p->Q = 7;
    p->Nx = prm->grid[0]; p->Ny = prm->grid[1]; p->Nz = prm->grid[2];
    p->Mx = 2 * p->Nx; p->My = 2 * p->Ny; p->Mz = 2 * p->Nz;
    p->large_plane = !plane_fits;
    p->Ng = int64_t(p->Nx) * p->Ny * p->Nz;
    const int64_t nt = m->nt, Q = p->Q;

    // ---- geometry
    std::vector<double> verts(9 * nt), area(nt), cen(3 * nt), diam(nt);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < m->nv; ++i)
        for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], m->xyz[3 * i + d]); hi[d] = std::max(hi[d], m->xyz[3 * i + d]); }
    double max_diam = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        for (int k = 0; k < 3; ++k)
            for (int d = 0; d < 3; ++d) verts[9 * t + 3 * k + d] = m->xyz[3 * m->tri[3 * t + k] + d];
        const double *v = &verts[9 * t];
        double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]}, e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        area[t] = 0.5 * std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int d = 0; d < 3; ++d) cen[3 * t + d] = (v[d] + v[3 + d] + v[6 + d]) / 3.0;
        double dm = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double *a = v + 3 * k, *b = v + 3 * ((k + 1) % 3);
            double x = b[0] - a[0], y = b[1] - a[1], z = b[2] - a[2];
            dm = std::max(dm, std::sqrt(x * x + y * y + z * z));
        }
        diam[t] = dm;
        max_diam = std::max(max_diam, dm);
    }
    p->tri_cen = cen;
    double max_h = 0.0;
    for (int d = 0; d < 3; ++d) {
        p->lo[d] = lo[d];
        p->h[d] = (hi[d] - lo[d]) / (prm->grid[d] - 1);
        if (!(p->h[d] > 0.0)) return bail(fail(SIE_ERR_ARG, "pfft_plan_create: mesh is flat along an axis"));
        max_h = std::max(max_h, p->h[d]);
    }
    p->r_near = std::max(prm->near_factor * max_h, prm->near_min_diam * max_diam);

    // ---- sample points, moments, stencils
    std::vector<double> r7b, r7w;
    radon7(r7b, r7w);
    const int64_t npt = nt * Q;
    std::vector<double> mom(9 * npt), lw(3 * O * npt);
    std::vector<int32_t> start(3 * npt);
    for (int64_t t = 0; t < nt; ++t) {
        const double *v = &verts[9 * t];
        for (int q = 0; q < Q; ++q) {
            const int64_t pt = t * Q + q;
            double r[3];
            for (int d = 0; d < 3; ++d) r[d] = r7b[3 * q] * v[d] + r7b[3 * q + 1] * v[3 + d] + r7b[3 * q + 2] * v[6 + d];
            for (int k = 0; k < 3; ++k)
                for (int d = 0; d < 3; ++d) mom[9 * pt + 3 * k + d] = 0.5 * r7w[q] * (r[d] - v[3 * k + d]);
            for (int d = 0; d < 3; ++d) {
                const int n = prm->grid[d];
                double tt = (r[d] - p->lo[d]) / p->h[d];
                long s0 = (O % 2) ? long(std::floor(tt + 0.5)) - (O - 1) / 2 : long(std::floor(tt)) - (O / 2 - 1);
                s0 = std::min<long>(std::max<long>(s0, 0), n - O);
                start[3 * pt + d] = int32_t(s0);
                for (int i = 0; i < O; ++i) {
                    double wv = 1.0;
                    for (int j = 0; j < O; ++j)
                        if (j != i) wv *= (tt - double(s0 + j)) / double(i - j);
                    lw[(3 * pt + d) * O + i] = wv;
                }
            }
        }
    }
    // ---- projection blocks (Sec. IV-B step 1 with the point currents folded in):
    // W(n, T)[d][k] = sum over T's points q whose stencil holds n of
    // L_n(r_q) (w_q/2)(r_q - v_k)_d, so that the grid current at node n is
    // Q_g[d][n] = sum_T sum_k W(n, T)[d][k] c_T[k], and the interpolated
    // far-field potential of triangle T is sum_n sum_d W(n, T)[d][k] phi_g[d][n].
    const int O3 = O * O * O;
    std::vector<int64_t> pt_ptr(nt + 1, 0);
    std::vector<int32_t> pt_node;
    std::vector<double> pt_W;   // [pair][3][3] as W[d][k]
    pt_node.reserve(size_t(nt) * 64);
    pt_W.reserve(size_t(nt) * 64 * 9);
    {
        struct Item { int64_t node; int q; double w; };
        std::vector<Item> items(size_t(Q) * O3);
        for (int64_t t = 0; t < nt; ++t) {
            size_t at = 0;
            for (int q = 0; q < Q; ++q) {
                const int64_t pt = t * Q + q;
                for (int i = 0; i < O; ++i)
                    for (int j = 0; j < O; ++j)
                        for (int k = 0; k < O; ++k) {
                            const int64_t node = (int64_t(start[3 * pt] + i) * p->Ny + (start[3 * pt + 1] + j)) * p->Nz +
                                                 (start[3 * pt + 2] + k);
                            const double w = (lw[(3 * pt) * O + i] * lw[(3 * pt + 1) * O + j]) * lw[(3 * pt + 2) * O + k];
                            items[at++] = Item{node, q, w};
                        }
            }
            // nodes ascending; per node the points in ascending order
            std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.node < b.node; });
            for (size_t a = 0; a < items.size();) {
                size_t b = a;
                double W[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                for (; b < items.size() && items[b].node == items[a].node; ++b) {
                    const double *mq = &mom[9 * (t * Q + items[b].q)];   // [k][d]
                    for (int d = 0; d < 3; ++d)
                        for (int k = 0; k < 3; ++k) W[3 * d + k] += items[b].w * mq[3 * k + d];
                }
                pt_node.push_back(int32_t(items[a].node));
                pt_W.insert(pt_W.end(), W, W + 9);
                a = b;
            }
            pt_ptr[t + 1] = int64_t(pt_node.size());
        }
    }
    const int64_t n_pair = int64_t(pt_node.size());
    p->n_pair = n_pair;
    // the same blocks by node (triangles ascending), and the 32-node tiles in use
    std::vector<int64_t> pn_ptr(p->Ng + 1, 0);
    for (int64_t e = 0; e < n_pair; ++e) pn_ptr[pt_node[e] + 1]++;
    for (int64_t i = 0; i < p->Ng; ++i) pn_ptr[i + 1] += pn_ptr[i];
    std::vector<Rec<double>> pn_rec64(n_pair), pt_rec64(n_pair);
    std::vector<Rec<float>> pn_rec32(n_pair), pt_rec32(n_pair);
    {
        std::vector<int64_t> fill(pn_ptr.begin(), pn_ptr.end() - 1);
        for (int64_t t = 0; t < nt; ++t)
            for (int64_t e = pt_ptr[t]; e < pt_ptr[t + 1]; ++e) {
                const double *W = &pt_W[9 * e];
                Rec<double> &a = pn_rec64[fill[pt_node[e]]++];
                Rec<double> &b = pt_rec64[e];
                a = Rec<double>{};
                b = Rec<double>{};
                for (int d = 0; d < 3; ++d)
                    for (int k = 0; k < 3; ++k) {
                        a.b[3 * d + k] = W[3 * d + k];   // out d, in k: grid current from c_T
                        b.b[3 * k + d] = W[3 * d + k];   // out k, in d: triangle potential from phi_g
                    }
                a.col = t;
                b.col = pt_node[e];
            }
        for (int64_t e = 0; e < n_pair; ++e) {
            pn_rec32[e] = Rec<float>{};
            pt_rec32[e] = Rec<float>{};
            for (int i = 0; i < 9; ++i) {
                pn_rec32[e].b[i] = float(pn_rec64[e].b[i]);
                pt_rec32[e].b[i] = float(pt_rec64[e].b[i]);
            }
            pn_rec32[e].col = int32_t(pn_rec64[e].col);
            pt_rec32[e].col = int32_t(pt_rec64[e].col);
        }
    }
    std::vector<int32_t> tiles;
    for (int64_t tl = 0; tl * 32 < p->Ng; ++tl)
        if (pn_ptr[std::min<int64_t>(p->Ng, tl * 32 + 32)] > pn_ptr[tl * 32]) tiles.push_back(int32_t(tl));
    p->n_tiles = int64_t(tiles.size());
    // projection chunks: node tiles of 2 x 4 x 8 (x, y, z), nodes ascending, cut
    // where the next node's triangles would take the chunk past kChunkTri; the
    // local index of each node record's triangle in its chunk.  A node touching
    // more than kChunkTri triangles leaves the plan on the direct projection.
    std::vector<int32_t> pch_node_ptr{0}, pch_nodes, pch_tri_ptr{0}, pch_tri;
    std::vector<uint16_t> pn_lcol(size_t(std::max<int64_t>(n_pair, 1)), 0);
    bool chunks_ok = true;
    for (int64_t n = 0; n < p->Ng && chunks_ok; ++n) chunks_ok = pn_ptr[n + 1] - pn_ptr[n] <= kChunkTri;
    if (chunks_ok) {
        std::vector<int64_t> stamp(nt, -1);
        std::vector<int32_t> local(nt, 0);
        int64_t chunk = 0;
        int32_t ntri = 0;
        auto close = [&]() {
            if (int64_t(pch_nodes.size()) == pch_node_ptr.back()) return;
            pch_node_ptr.push_back(int32_t(pch_nodes.size()));
            pch_tri_ptr.push_back(int32_t(pch_tri.size()));
            ++chunk;
            ntri = 0;
        };
        for (int x0 = 0; x0 < p->Nx; x0 += 2)
            for (int y0 = 0; y0 < p->Ny; y0 += 4)
                for (int z0 = 0; z0 < p->Nz; z0 += 8) {
                    for (int x = x0; x < std::min(x0 + 2, p->Nx); ++x)
                        for (int y = y0; y < std::min(y0 + 4, p->Ny); ++y)
                            for (int z = z0; z < std::min(z0 + 8, p->Nz); ++z) {
                                const int64_t n = (int64_t(x) * p->Ny + y) * p->Nz + z;
                                int32_t fresh = 0;
                                for (int64_t e = pn_ptr[n]; e < pn_ptr[n + 1]; ++e)
                                    fresh += stamp[pn_rec64[e].col] != chunk;
                                if (ntri + fresh > kChunkTri) close();
                                for (int64_t e = pn_ptr[n]; e < pn_ptr[n + 1]; ++e) {
                                    const int64_t t = pn_rec64[e].col;
                                    if (stamp[t] != chunk) {
                                        stamp[t] = chunk;
                                        local[t] = ntri++;
                                        pch_tri.push_back(int32_t(t));
                                    }
                                    pn_lcol[e] = uint16_t(local[t]);
                                }
                                pch_nodes.push_back(int32_t(n));
                            }
                    close();
                }
    }
    p->n_pchunk = chunks_ok ? int64_t(pch_node_ptr.size()) - 1 : 0;
    // ---- near list (exact criterion per pair; a cell list only prunes candidates)
    std::vector<int32_t> bmin(3 * nt), bmax(3 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int d = 0; d < 3; ++d) {
            int32_t a = INT32_MAX, b = INT32_MIN;
            for (int q = 0; q < Q; ++q) { a = std::min(a, start[3 * (t * Q + q) + d]); b = std::max(b, start[3 * (t * Q + q) + d]); }
            bmin[3 * t + d] = a;
            bmax[3 * t + d] = b + O - 1;
        }
    const double rc = std::max(p->r_near, 2.0 * max_diam + (O + 1) * max_h);
    int nc[3];
    for (int d = 0; d < 3; ++d) nc[d] = std::max(1, int(std::min(1024.0, std::floor((hi[d] - lo[d]) / rc) + 1)));
    std::vector<int64_t> cell_ptr(int64_t(nc[0]) * nc[1] * nc[2] + 1, 0);
    auto cell_of = [&](int64_t t, int d) { return std::min(nc[d] - 1, int((cen[3 * t + d] - lo[d]) / rc)); };
    std::vector<int64_t> tcell(nt);
    for (int64_t t = 0; t < nt; ++t) {
        tcell[t] = (int64_t(cell_of(t, 0)) * nc[1] + cell_of(t, 1)) * nc[2] + cell_of(t, 2);
        cell_ptr[tcell[t] + 1]++;
    }
    for (size_t i = 0; i + 1 < cell_ptr.size(); ++i) cell_ptr[i + 1] += cell_ptr[i];
    std::vector<int32_t> cell_tri(nt);
    {
        std::vector<int64_t> f(cell_ptr.begin(), cell_ptr.end() - 1);
        for (int64_t t = 0; t < nt; ++t) cell_tri[f[tcell[t]]++] = int32_t(t);
    }
    const double r2 = p->r_near * p->r_near;
    std::vector<std::vector<int32_t>> rows(nt);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nt; ++t) {
        int cx = cell_of(t, 0), cy = cell_of(t, 1), cz = cell_of(t, 2);
        auto &row = rows[t];
        for (int ix = std::max(0, cx - 1); ix <= std::min(nc[0] - 1, cx + 1); ++ix)
            for (int iy = std::max(0, cy - 1); iy <= std::min(nc[1] - 1, cy + 1); ++iy)
                for (int iz = std::max(0, cz - 1); iz <= std::min(nc[2] - 1, cz + 1); ++iz) {
                    int64_t c = (int64_t(ix) * nc[1] + iy) * nc[2] + iz;
                    for (int64_t k = cell_ptr[c]; k < cell_ptr[c + 1]; ++k) {
                        int64_t j = cell_tri[k];
                        double dx = cen[3 * j] - cen[3 * t], dy = cen[3 * j + 1] - cen[3 * t + 1], dz = cen[3 * j + 2] - cen[3 * t + 2];
                        double d2 = dx * dx + dy * dy + dz * dz;
                        bool box = true;
                        for (int d = 0; d < 3; ++d)
                            box = box && bmin[3 * j + d] <= bmax[3 * t + d] && bmax[3 * j + d] >= bmin[3 * t + d];
                        if (d2 < r2 || box) row.push_back(int32_t(j));
                    }
                }
        std::sort(row.begin(), row.end());
    }
    std::vector<int64_t> near_ptr(nt + 1, 0);
    for (int64_t t = 0; t < nt; ++t) near_ptr[t + 1] = near_ptr[t] + int64_t(rows[t].size());
    p->n_near = near_ptr[nt];
    std::vector<int32_t> near_col(p->n_near);
    for (int64_t t = 0; t < nt; ++t) std::copy(rows[t].begin(), rows[t].end(), near_col.begin() + near_ptr[t]);
    rows.clear();
    rows.shrink_to_fit();

    // ---- Gram blocks, per-triangle branch maps
    std::vector<double> gram(9 * nt);
    for (int64_t t = 0; t < nt; ++t) {
        const double *v = &verts[9 * t];
        double s[3] = {v[0] + v[3] + v[6], v[1] + v[4] + v[7], v[2] + v[5] + v[8]};
        double c[3] = {s[0] / 3.0, s[1] / 3.0, s[2] / 3.0};
        double quad = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3] + v[4] * v[4] + v[5] * v[5] +
                       v[6] * v[6] + v[7] * v[7] + v[8] * v[8] + s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) / 12.0;
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
                const double *a = v + 3 * k, *b = v + 3 * l;
                double ac = a[0] * c[0] + a[1] * c[1] + a[2] * c[2], bc = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
                double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
                gram[9 * t + 3 * k + l] = (quad - ac - bc + ab) / (4.0 * area[t]);
            }
    }
    std::vector<int32_t> tb(3 * nt, -1), cond(m->cond.begin(), m->cond.end());
    std::vector<int8_t> ts(3 * nt, 0);
    std::vector<double> diag_gram(L->nb, 0.0);
    std::vector<int32_t> br_cond(L->nb), twig_node(L->nb, -1);
    for (int64_t b = 0; b < L->nb; ++b) {
        for (int s = 0; s < 2; ++s) {
            int32_t t = L->br_tri[2 * b + s];
            int k = L->br_local[2 * b + s];
            tb[3 * t + k] = int32_t(b);
            ts[3 * t + k] = s ? -1 : 1;
            diag_gram[b] += gram[9 * t + 4 * k];
        }
        br_cond[b] = m->cond[L->br_tri[2 * b]];
    }
    for (int64_t v = 0; v < L->n_nodes; ++v)
        if (L->parent_branch[v] >= 0) twig_node[L->parent_branch[v]] = int32_t(v);

    // ---- uploads
    int rcode;
#define UP(dst, src) do { if ((rcode = upload(p, &(dst), src))) return bail(rcode); } while (0)
    UP(p->d_tb, tb);
    UP(p->d_ts, ts);
    UP(p->d_cond, cond);
    UP(p->d_gram, gram);
    UP(p->d_mom64, mom);
    UP(p->d_mom32, to_f32(mom));
    UP(p->d_start, start);
    UP(p->d_lw64, lw);
    UP(p->d_lw32, to_f32(lw));
    UP(p->d_pn_ptr, pn_ptr);
    UP(p->d_pn_rec64, pn_rec64);
    UP(p->d_pn_rec32, pn_rec32);
    UP(p->d_pt_ptr, pt_ptr);
    UP(p->d_pt_rec64, pt_rec64);
    UP(p->d_pt_rec32, pt_rec32);
    UP(p->d_tiles, tiles);
    if (p->n_pchunk > 0) {
        UP(p->d_pch_node_ptr, pch_node_ptr);
        UP(p->d_pch_nodes, pch_nodes);
        UP(p->d_pch_tri_ptr, pch_tri_ptr);
        UP(p->d_pch_tri, pch_tri);
        UP(p->d_pn_lcol, pn_lcol);
    }
    UP(p->d_near_ptr, near_ptr);
    UP(p->d_near_col, near_col);
    {
        std::vector<int32_t> tn(L->tour_node.begin(), L->tour_node.end());
        UP(p->d_tour_node, tn);
        std::vector<int8_t> te(L->tour_is_enter.begin(), L->tour_is_enter.end());
        UP(p->d_tour_enter, te);
        std::vector<int32_t> en(L->enter.begin(), L->enter.end()), ex(L->exit_.begin(), L->exit_.end());
        UP(p->d_enter, en);
        UP(p->d_exit, ex);
        std::vector<int32_t> np_(L->nl_ptr.begin(), L->nl_ptr.end()), nlo(L->nl_loop.begin(), L->nl_loop.end());
        std::vector<int8_t> nls(L->nl_sign.begin(), L->nl_sign.end());
        UP(p->d_nl_ptr, np_);
        UP(p->d_nl_loop, nlo);
        UP(p->d_nl_sign, nls);
        std::vector<int32_t> pb(L->parent_branch.begin(), L->parent_branch.end());
        UP(p->d_parent_branch, pb);
        // reference node of each part: the sink contact of its first port, else its tree root
        std::vector<int64_t> ref(L->n_comp, -1);
        for (size_t q = 0; q < L->port_sink.size(); ++q) {
            const int32_t v = L->port_sink[q];
            if (ref[L->comp[v]] < 0) ref[L->comp[v]] = v;
        }
        for (int64_t v = 0; v < L->n_nodes; ++v)
            if (L->parent[v] < 0 && ref[L->comp[v]] < 0) ref[L->comp[v]] = v;
        std::vector<int32_t> ps(nt), pr(nt);
        for (int64_t t = 0; t < nt; ++t) {
            const int64_t v = L->node_of_tri[t];
            ps[t] = L->enter[v];
            pr[t] = L->enter[ref[L->comp[v]]];
        }
        UP(p->d_panel_slot, ps);
        UP(p->d_panel_ref, pr);
        UP(p->d_twig_node, twig_node);
        std::vector<int32_t> lob(L->loop_of_branch.begin(), L->loop_of_branch.end());
        UP(p->d_loop_of_branch, lob);
        std::vector<int32_t> ta(L->tail.begin(), L->tail.end()), he(L->head.begin(), L->head.end());
        UP(p->d_tail, ta);
        UP(p->d_head, he);
        std::vector<int32_t> lb(L->link_branch.begin(), L->link_branch.end());
        UP(p->d_link_branch, lb);
        std::vector<int32_t> bt(L->br_tri.begin(), L->br_tri.end());
        UP(p->d_br_tri, bt);
        std::vector<int8_t> bl(L->br_local.begin(), L->br_local.end());
        UP(p->d_br_local, bl);
    }
    UP(p->d_diag_gram, diag_gram);
    UP(p->d_br_cond, br_cond);
    // twiddles
    for (int a = 0; a < 3; ++a) {
        const int M = 2 * prm->grid[a];
        std::vector<double2> w64(M);
        std::vector<float2> w32(M);
        for (int k = 0; k < M; ++k) {
            double ang = 2.0 * M_PI * double(k) / double(M);
            w64[k] = make_double2(std::cos(ang), -std::sin(ang));
            w32[k] = make_float2(float(w64[k].x), float(w64[k].y));
        }
        UP(p->d_tw64[a], w64);
        UP(p->d_tw32[a], w32);
        int n1, n2;
        split4(M, n1, n2);
        std::vector<double2> tf(M), ti(M);
        std::vector<float2> tf32(M), ti32(M);
        for (int j2 = 0; j2 < n2; ++j2)
            for (int k1 = 0; k1 < n1; ++k1) {
                tf[j2 * n1 + k1] = w64[(j2 * k1) % M];
                ti[k1 * n2 + j2] = w64[(j2 * k1) % M];
            }
        for (int k = 0; k < M; ++k) {
            tf32[k] = make_float2(float(tf[k].x), float(tf[k].y));
            ti32[k] = make_float2(float(ti[k].x), float(ti[k].y));
        }
        UP(p->d_tf64[a], tf);
        UP(p->d_ti64[a], ti);
        UP(p->d_tf32[a], tf32);
        UP(p->d_ti32[a], ti32);
    }
    // device-side geometry for the setup kernels
    double *d_verts = nullptr, *d_area = nullptr, *d_r7b = nullptr, *d_r7w = nullptr, *d_tgb = nullptr, *d_tgw = nullptr;
    int32_t *d_tri = nullptr;
    std::vector<double> tgb, tgw;
    collapsed_gauss(prm->n_touch, tgb, tgw);
    std::vector<int32_t> tri(m->tri.begin(), m->tri.end());
    UP(d_verts, verts);
    UP(d_area, area);
    UP(d_r7b, r7b);
    UP(d_r7w, r7w);
    UP(d_tgb, tgb);
    UP(d_tgw, tgw);
    UP(d_tri, tri);
#undef UP
    cudaStream_t s = p->stream;
    // ---- kernel table and spectrum (FP64)
    const int64_t nM = int64_t(p->Mx) * p->My * p->Mz;
    double *d_Hpad = nullptr;
    double2 *d_Hc = nullptr;
    if ((rcode = plan_alloc(p, (void **)&d_Hpad, nM * sizeof(double)))) return bail(rcode);
    if ((rcode = plan_alloc(p, (void **)&d_Hc, nM * sizeof(double2)))) return bail(rcode);
    k_fill_kernel<<<(nM + 255) / 256, 256, 0, s>>>(d_Hpad, d_Hc, p->Mx, p->My, p->Mz, p->h[0], p->h[1], p->h[2], prm->h0);
    p->launches++;
    {
        double2 *d_spec = nullptr;
        if ((rcode = kernel_fft3(p, d_Hc, &d_spec, s))) return bail(rcode);
        SIE_CUDA(cudaStreamSynchronize(s));
        if (d_spec != d_Hc) {
            plan_free(p, d_Hc);
            d_Hc = d_spec;
        }
        const int64_t nh = int64_t(p->Mx / 2 + 1) * (p->My / 2 + 1) * (p->Mz / 2 + 1);
        if ((rcode = plan_alloc(p, (void **)&p->d_H64, nh * sizeof(double)))) return bail(rcode);
        if ((rcode = plan_alloc(p, (void **)&p->d_H32, nh * sizeof(float)))) return bail(rcode);
        k_extract_H<<<(nh + 255) / 256, 256, 0, s>>>(d_Hc, p->d_H64, p->d_H32, p->Mx, p->My, p->Mz, 1.0 / double(nM));
        p->launches++;
        if ((rcode = plan_alloc(p, (void **)&p->d_Hp64, nh * sizeof(double)))) return bail(rcode);
        if ((rcode = plan_alloc(p, (void **)&p->d_Hp32, nh * sizeof(float)))) return bail(rcode);
        k_permute_H<<<(nh + 255) / 256, 256, 0, s>>>(p->d_H64, p->d_Hp64, p->d_Hp32, p->Mx / 2 + 1, p->My / 2 + 1,
                                                     p->Mz / 2 + 1);
        p->launches++;
    }
    // ---- near-field blocks
    if ((rcode = plan_alloc(p, (void **)&p->d_Ldir64, p->n_near * 9 * sizeof(double)))) return bail(rcode);
    if ((rcode = plan_alloc(p, (void **)&p->d_Ld64, p->n_near * 9 * sizeof(double)))) return bail(rcode);
    if ((rcode = plan_alloc(p, (void **)&p->d_near_rec64, p->n_near * sizeof(Rec<double>)))) return bail(rcode);
    if ((rcode = plan_alloc(p, (void **)&p->d_near_rec32, p->n_near * sizeof(Rec<float>)))) return bail(rcode);
    {
        NearArgs a{p->d_near_ptr, p->d_near_col, nt, d_verts, d_area, d_tri, d_r7b, d_r7w, d_tgb, d_tgw,
                   int(tgw.size()), p->d_start, p->d_lw64, p->d_mom64, d_Hpad, int(Q), O, p->Mx, p->My, p->Mz,
                   p->d_Ldir64, p->d_Ld64};
        k_near_blocks<<<(p->n_near + 127) / 128, 128, 0, s>>>(a, p->n_near);
        p->launches++;
    }
    SIE_CUDA(cudaGetLastError());
    k_pack_near<<<(p->n_near + 255) / 256, 256, 0, s>>>(p->d_near_col, p->d_Ld64, p->n_near, p->d_near_rec64,
                                                         p->d_near_rec32);
    p->launches++;
    if ((rcode = near_mma_prepare(p, near_ptr, near_col, s))) return bail(rcode);
    if ((rcode = plan_alloc(p, (void **)&p->d_err, sizeof(int)))) return bail(rcode);
    SIE_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
    if (cudaMallocHost((void **)&p->h_err, sizeof(int)) != cudaSuccess) p->h_err = nullptr;   // optional
    else *p->h_err = 0;
    if ((rcode = plan_alloc(p, (void **)&p->d_diag_L, L->nb * sizeof(double)))) return bail(rcode);
    k_branch_diag<<<(L->nb + 255) / 256, 256, 0, s>>>(p->d_near_ptr, p->d_near_col, p->d_Ldir64, p->d_br_tri,
                                                      p->d_br_local, L->nb, p->d_diag_L);
    p->launches++;
    SIE_CUDA(cudaGetLastError());
    SIE_CUDA(cudaStreamSynchronize(s));
    if (prm->kernel == SIE_KERNEL_LOSSY) {
        // the per-frequency near blocks of the lossy kernel are built from the vertices
        // and the Radon rule on first use of each frequency
        p->d_verts = d_verts;
        p->d_r7b = d_r7b;
        p->d_r7w = d_r7w;
        d_verts = d_r7b = d_r7w = nullptr;
    }
    for (void *tmp : {(void *)d_Hpad, (void *)d_Hc, (void *)d_verts, (void *)d_area, (void *)d_r7b, (void *)d_r7w,
                      (void *)d_tgb, (void *)d_tgw, (void *)d_tri})
        if (tmp) plan_free(p, tmp);
    *out = p;
    return SIE_OK;
}

extern "C" void pfft_plan_destroy(pfft_plan *p) {
    if (!p) return;
    sie::plan_free_precond(p);
    sie::plan_free_lossy(p);
    for (auto &e : p->prof_pending) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (void *a : p->allocations) cudaFree(a);
    if (p->h_err) cudaFreeHost(p->h_err);
    if (p->pool) {
        cudaDeviceSynchronize();   // stream-ordered frees of the solve path have completed
        cudaMemPoolDestroy(p->pool);
    }
    for (void *a : {p->scr.tour, p->scr.grid, p->scr.spec, p->scr.phiT, p->scr.y_tri, p->scr.y_br,
                    (void *)p->scr.coef, p->scr.cT, p->scr.ffar})
        if (a) cudaFree(a);
    delete p;
}

extern "C" int pfft_plan_info(const pfft_plan *p, int64_t *n_loops, int64_t *n_branches, int64_t *n_tri,
                              int64_t *n_near_pairs, double *grid_h, double *r_near, int64_t *device_bytes) {
    if (!p) return fail(SIE_ERR_ARG, "pfft_plan_info: NULL plan");
    if (n_loops) *n_loops = p->nl;
    if (n_branches) *n_branches = p->nb;
    if (n_tri) *n_tri = p->nt;
    if (n_near_pairs) *n_near_pairs = p->n_near;
    if (grid_h) for (int d = 0; d < 3; ++d) grid_h[d] = p->h[d];
    if (r_near) *r_near = p->r_near;
    if (device_bytes) *device_bytes = int64_t(p->device_bytes + p->scr.bytes);
    return SIE_OK;
}

extern "C" int pfft_plan_export(const pfft_plan *p, int32_t what, void *host_out, int64_t capacity_bytes) {
    if (!p || !host_out) return fail(SIE_ERR_ARG, "pfft_plan_export: NULL argument");
    const void *src = nullptr;
    int64_t bytes = 0;
    switch (what) {
        case SIE_EXPORT_NEAR_PTR: src = p->d_near_ptr; bytes = (p->nt + 1) * 8; break;
        case SIE_EXPORT_NEAR_COL: src = p->d_near_col; bytes = p->n_near * 4; break;
        case SIE_EXPORT_LD: src = p->d_Ld64; bytes = p->n_near * 72; break;
        case SIE_EXPORT_LDIRECT: src = p->d_Ldir64; bytes = p->n_near * 72; break;
        case SIE_EXPORT_HHAT: src = p->d_H64; bytes = int64_t(p->Nx + 1) * (p->Ny + 1) * (p->Nz + 1) * 8; break;
        case SIE_EXPORT_START: src = p->d_start; bytes = p->nt * p->Q * 3 * 4; break;
        case SIE_EXPORT_PROJ_PTR: src = p->d_pt_ptr; bytes = (p->nt + 1) * 8; break;
        case SIE_EXPORT_PROJ_NODE:
        case SIE_EXPORT_PROJ_W: {
            // unpacked from the per-triangle records {b[3k + d] = W[d][k], col = n}
            bytes = p->n_pair * (what == SIE_EXPORT_PROJ_NODE ? 4 : 72);
            if (capacity_bytes < bytes) return fail(SIE_ERR_ARG, "pfft_plan_export: buffer too small");
            std::vector<Rec<double>> rec(size_t(p->n_pair));
            SIE_CUDA(cudaMemcpy(rec.data(), p->d_pt_rec64, rec.size() * sizeof(Rec<double>), cudaMemcpyDeviceToHost));
            for (int64_t e = 0; e < p->n_pair; ++e) {
                if (what == SIE_EXPORT_PROJ_NODE) {
                    static_cast<int32_t *>(host_out)[e] = int32_t(rec[e].col);
                } else {
                    double *W = static_cast<double *>(host_out) + 9 * e;
                    for (int d = 0; d < 3; ++d)
                        for (int k = 0; k < 3; ++k) W[3 * d + k] = rec[e].b[3 * k + d];
                }
            }
            return SIE_OK;
        }
        default: return fail(SIE_ERR_ARG, "pfft_plan_export: unknown array");
    }
    if (capacity_bytes < bytes) return fail(SIE_ERR_ARG, "pfft_plan_export: buffer too small");
    SIE_CUDA(cudaMemcpy(host_out, src, size_t(bytes), cudaMemcpyDeviceToHost));
    return SIE_OK;
}

extern "C" int pfft_convolve(pfft_plan *p, void *grid, int32_t nbatch, int32_t prec, void *cuda_stream) {
    if (!p || !grid || nbatch < 1) return fail(SIE_ERR_ARG, "pfft_convolve: bad argument");
    if (prec != SIE_PREC_FP64 && prec != SIE_PREC_MIXED) return fail(SIE_ERR_ARG, "pfft_convolve: bad precision");
    const int32_t R = (nbatch + 2) / 3;
    int rc = scratch_reserve(p, R, prec);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // fft_conv works on 3R grids; run it on the caller's nbatch grids by
    // treating them as ceil(nbatch/3) groups when nbatch is a multiple of 3,
    // else one grid at a time through the scratch spectrum.
    if (nbatch % 3 == 0) {
        rc = fft_conv(p, grid, p->scr.spec, R, prec, s);
    } else {
        const size_t gb = size_t(p->Ng) * (prec == SIE_PREC_FP64 ? 16 : 8);
        for (int32_t b = 0; b < nbatch && !rc; ++b) rc = fft_conv_n(p, (char *)grid + b * gb, p->scr.spec, 1, prec, s);
    }
    if (rc) return rc;
    SIE_CUDA(cudaStreamSynchronize(s));
    return SIE_OK;
}

namespace sie {
int lossy_fill_table(pfft_plan *p, double inv_delta, double2 *Hc, cudaStream_t s) {
    const int64_t nM = int64_t(p->Mx) * p->My * p->Mz;
    k_fill_kernel_lossy<<<unsigned((nM + 255) / 256), 256, 0, s>>>(Hc, p->Mx, p->My, p->Mz, p->h[0], p->h[1], p->h[2],
                                                                   p->params.h0, inv_delta);
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

int lossy_table_spectrum(pfft_plan *p, double2 *Hc, double2 *H64, float2 *H32, cudaStream_t s) {
    const int64_t nM = int64_t(p->Mx) * p->My * p->Mz;
    const int64_t nh = int64_t(p->Mx / 2 + 1) * (p->My / 2 + 1) * (p->Mz / 2 + 1);
    double2 *spec = nullptr;
    int rc = kernel_fft3(p, Hc, &spec, s);
    if (rc) return rc;
    k_extract_Hc<<<unsigned((nh + 255) / 256), 256, 0, s>>>(spec, H64, H32, p->Mx, p->My, p->Mz, 1.0 / double(nM));
    p->launches++;
    const cudaError_t e = cudaGetLastError();
    if (spec != Hc) {
        cudaStreamSynchronize(s);
        plan_free(p, spec);
    }
    if (e != cudaSuccess) return fail(SIE_ERR_CUDA, std::string("lossy spectrum: ") + cudaGetErrorString(e));
    return SIE_OK;
}

// Spectrum of the lossy kernel for (omega, sigma), kept until another pair is asked for.
int lossy_spectrum(pfft_plan *p, double omega, double sigma, cudaStream_t s) {
    if (p->d_Hl64 && p->lossy_omega == omega && p->lossy_sigma == sigma) return SIE_OK;
    const int64_t nM = int64_t(p->Mx) * p->My * p->Mz;
    const int64_t nh = int64_t(p->Mx / 2 + 1) * (p->My / 2 + 1) * (p->Mz / 2 + 1);
    int rc;
    if (!p->d_Hl64) {
        if ((rc = plan_alloc(p, (void **)&p->d_Hl64, nh * sizeof(double2)))) return rc;
        if ((rc = plan_alloc(p, (void **)&p->d_Hl32, nh * sizeof(float2)))) return rc;
    }
    double2 *d_Hc = nullptr, *d_Hc2 = nullptr;
    if ((rc = plan_alloc(p, (void **)&d_Hc, nM * sizeof(double2)))) return rc;
    auto done = [&](int r) {
        if (d_Hc2 && d_Hc2 != d_Hc) plan_free(p, d_Hc2);
        plan_free(p, d_Hc);
        return r;
    };
    const double mu0 = 4e-7 * M_PI;
    const double inv_delta = std::sqrt(omega * mu0 * sigma / 2.0);   // 1/delta, delta the skin depth
    k_fill_kernel_lossy<<<unsigned((nM + 255) / 256), 256, 0, s>>>(d_Hc, p->Mx, p->My, p->Mz, p->h[0], p->h[1],
                                                                   p->h[2], p->params.h0, inv_delta);
    p->launches++;
    if ((rc = kernel_fft3(p, d_Hc, &d_Hc2, s))) return done(rc);
    k_extract_Hc<<<unsigned((nh + 255) / 256), 256, 0, s>>>(d_Hc2, p->d_Hl64, p->d_Hl32, p->Mx, p->My, p->Mz,
                                                          1.0 / double(nM));
    p->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(fail(SIE_ERR_CUDA, std::string("lossy spectrum: ") + cudaGetErrorString(e)));
    p->lossy_omega = omega;
    p->lossy_sigma = sigma;
    return done(SIE_OK);
}
}  // namespace sie

extern "C" int pfft_convolve_lossy(pfft_plan *p, void *grid, int32_t nbatch, double omega, double sigma, int32_t prec,
                                   void *cuda_stream) {
    if (!p || !grid || nbatch < 1) return fail(SIE_ERR_ARG, "pfft_convolve_lossy: bad argument");
    if (prec != SIE_PREC_FP64 && prec != SIE_PREC_MIXED) return fail(SIE_ERR_ARG, "pfft_convolve_lossy: bad precision");
    if (!(omega > 0.0) || !std::isfinite(omega) || !(sigma > 0.0) || !std::isfinite(sigma))
        return fail(SIE_ERR_ARG, "pfft_convolve_lossy: omega and sigma must be finite and > 0");
    (void)cudaGetLastError();
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int rc = lossy_spectrum(p, omega, sigma, s);
    if (rc) return rc;
    rc = scratch_reserve(p, (nbatch + 2) / 3, prec);   // its x-transform buffer holds 3 grids per right-hand side
    if (rc) return rc;
    rc = fft_conv_n(p, grid, p->scr.spec, nbatch, prec, s, true);
    if (rc) return rc;
    SIE_CUDA(cudaStreamSynchronize(s));
    return SIE_OK;
}

extern "C" int pfft_profile_enable(pfft_plan *p, int32_t on) {
    if (!p) return fail(SIE_ERR_ARG, "pfft_profile_enable: NULL plan");
    for (auto &e : p->prof_pending) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    p->prof_pending.clear();
    for (int i = 0; i < SIE_NSTAGES; ++i) { p->prof_ms[i] = 0.0; p->prof_count[i] = 0; }
    p->prof_on = on != 0;
    return SIE_OK;
}

extern "C" int pfft_profile_read(pfft_plan *p, double *ms, int64_t *launches) {
    if (!p) return fail(SIE_ERR_ARG, "pfft_profile_read: NULL plan");
    for (auto &e : p->prof_pending) {
        SIE_CUDA(cudaEventSynchronize(e.b));
        float t = 0.f;
        SIE_CUDA(cudaEventElapsedTime(&t, e.a, e.b));
        p->prof_ms[e.stage] += t;
        p->prof_count[e.stage] += 1;
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    p->prof_pending.clear();
    for (int i = 0; i < SIE_NSTAGES; ++i) {
        if (ms) ms[i] = p->prof_ms[i];
        if (launches) launches[i] = p->prof_count[i];
    }
    return SIE_OK;
}

extern "C" int64_t pfft_plan_launches(const pfft_plan *p) { return p ? p->launches : 0; }
