// pfft_matvec: the loop-space product of Eq. (FinalME) with the inductive part
// applied by the pre-corrected FFT (Sec. IV-A, IV-B of arXiv 2210.04891):
//
//   alpha = A^T x                     (Eq. CurT; Euler-tour subtree sums)
//   J_q   = sum_k s_k alpha_k (w_q/2)(r_q - v_k)   point currents (Eq. RWG)
//   Q_g   = B alpha                   (Eq. Projection; node gather lists)
//   phi_g = H Q_g                     (Eq. FFTCal; zero-padded FFT convolution)
//   Phi_q = sum_n L_n(r_q) phi_n      (Eq. interpolation, I = B^T)
//   y_T   = Z_s G_T c_T + c_L (far_T + sum_T' L_d(T,T') c_T')    (Eq. Zb, Eq. Lb)
//   y     = A y_b                     (Eq. VolT; Euler-tour root-path sums)
//
// A^T x: the current of a twig equals minus the current its subtree receives
// through links (Kirchhoff's current law), a subtree sum = a difference of two
// prefix sums along the Euler tour.  A y: the voltage of a fundamental loop is
// its link's voltage plus psi(head) - psi(tail), psi(v) the sum of twig
// voltages on v's path to the root = a prefix sum of +-delta over the tour.
// Both are exact rewrites of the sparse products (no approximation).
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "sie_plan.h"

using namespace sie;

namespace {

constexpr double kMu0 = 4e-7 * M_PI;

template <typename V> __device__ __forceinline__ V shfl_up(V v, int d) {
    V o;
    o.x = __shfl_up_sync(0xffffffffu, v.x, d);
    o.y = __shfl_up_sync(0xffffffffu, v.y, d);
    return o;
}

// Inclusive prefix sum of each row (complex128) of a [R][n] array, in place.
// One CTA of 1024 threads per row, 4 items per thread per chunk.
__global__ void __launch_bounds__(1024) k_scan_rows(double2 *buf, int64_t n) {
    __shared__ double2 warp_tot[32];
    __shared__ double2 carry_s;
    double2 *row = buf + blockIdx.x * n;
    double2 carry = make_double2(0.0, 0.0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < n; base += 4 * 1024) {
        double2 v[4];
        double2 run = make_double2(0.0, 0.0);
        const int64_t i0 = base + 4 * int64_t(threadIdx.x);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (i0 + k < n) ? row[i0 + k] : make_double2(0.0, 0.0);
            run = cadd(run, v[k]);
            v[k] = run;
        }
        double2 incl = run;   // warp inclusive scan of thread totals
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            double2 o = shfl_up(incl, d);
            if (lane >= d) incl = cadd(incl, o);
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            double2 w = warp_tot[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                double2 o = shfl_up(w, d);
                if (lane >= d) w = cadd(w, o);
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        double2 off = carry;
        if (warp > 0) off = cadd(off, warp_tot[warp - 1]);
        off = cadd(off, csub(incl, run));   // exclusive within the warp
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k < n) row[i0 + k] = cadd(v[k], off);
        if (threadIdx.x == 1023) carry_s = cadd(off, run);
        __syncthreads();
        carry = carry_s;
        __syncthreads();
    }
}

// Tour values for A^T: at node v's enter slot the current the links inject
// into v (+x on links entering v, -x on links leaving it); 0 at exit slots.
__global__ void k_tour_inject(const double2 *__restrict__ x, int64_t nl, double2 *__restrict__ tour, int64_t nslots,
                              const int32_t *__restrict__ tour_node, const int8_t *__restrict__ tour_enter,
                              const int32_t *__restrict__ nl_ptr, const int32_t *__restrict__ nl_loop,
                              const int8_t *__restrict__ nl_sign, int32_t nrhs) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nslots * nrhs) return;
    int64_t r = i / nslots, s = i % nslots;
    double2 acc = make_double2(0.0, 0.0);
    if (tour_enter[s]) {
        int v = tour_node[s];
        for (int k = nl_ptr[v]; k < nl_ptr[v + 1]; ++k) {
            double2 xv = x[r * nl + nl_loop[k]];
            if (nl_sign[k] > 0) acc = cadd(acc, xv); else acc = csub(acc, xv);
        }
    }
    tour[i] = acc;
}

// Branch current of branch b for right-hand side r (loop space): a link carries
// its loop current; a twig above node v carries -sigma * (subtree inflow).
__device__ __forceinline__ double2 branch_current(int32_t b, int64_t r, const double2 *__restrict__ x, int64_t nl,
                                                  const double2 *__restrict__ P, int64_t nslots,
                                                  const int32_t *__restrict__ loop_of_branch,
                                                  const int32_t *__restrict__ twig_node, const int32_t *__restrict__ head,
                                                  const int32_t *__restrict__ enter, const int32_t *__restrict__ exit_) {
    int32_t l = loop_of_branch[b];
    if (l >= 0) return x[r * nl + l];
    int32_t v = twig_node[b];
    const double2 *row = P + r * nslots;
    double2 S = row[exit_[v]];
    int32_t e = enter[v];
    if (e > 0) S = csub(S, row[e - 1]);
    return head[b] == v ? mk<double>(-S.x, -S.y) : S;
}

template <typename T>
__global__ void k_alpha_tri(const double2 *__restrict__ x, int64_t nl, const double2 *__restrict__ P, int64_t nslots,
                            const int32_t *__restrict__ tb, const int8_t *__restrict__ ts,
                            const int32_t *__restrict__ loop_of_branch, const int32_t *__restrict__ twig_node,
                            const int32_t *__restrict__ head, const int32_t *__restrict__ enter,
                            const int32_t *__restrict__ exit_, int64_t nt, int32_t nrhs, int space, int64_t nb,
                            C<T> *__restrict__ c_tri, C<T> *__restrict__ cT) {
    // i = (t * 3 + k) * R + r: the RHS-innermost copy cT is written coalesced
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nt * 3 * nrhs) return;
    int64_t tk = i / nrhs, r = i % nrhs;
    int32_t b = tb[tk];
    double2 a = make_double2(0.0, 0.0);
    if (b >= 0) {
        if (space == SIE_SPACE_LOOP)
            a = branch_current(b, r, x, nl, P, nslots, loop_of_branch, twig_node, head, enter, exit_);
        else
            a = x[r * nb + b];
        if (ts[tk] < 0) { a.x = -a.x; a.y = -a.y; }
    }
    const C<T> v = mk<T>(T(a.x), T(a.y));
    cT[i] = v;
    c_tri[r * nt * 3 + tk] = v;
}

// Pre-corrected near field as a block-sparse x dense product (Eq. Lb):
// ynear[t][k][r] = sum_{t' near t} sum_l L_d(t, t')[k][l] cT[t'][l][r].
// One warp per (row t, chunk of 32 RB right-hand sides); each L_d block is read
// once per chunk and applied to all of its right-hand sides, lane r reading
// the neighbours' currents contiguously over r.
template <typename T, int RB>
__global__ void __launch_bounds__(256) k_near_spmm(const int64_t *__restrict__ near_ptr,
                                                   const int32_t *__restrict__ near_col, const T *__restrict__ Ld,
                                                   const C<T> *__restrict__ cT, int64_t nt, int32_t R, int32_t nchunk,
                                                   C<T> *__restrict__ ynear) {
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= nt * nchunk) return;
    const int64_t t = gw / nchunk;
    const int32_t r0 = int32_t(gw % nchunk) * 32 * RB + lane;
    C<T> acc[3][RB];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < RB; ++j) acc[k][j] = mk<T>(T(0), T(0));
    const int64_t e1 = near_ptr[t + 1];
#pragma unroll 2
    for (int64_t e = near_ptr[t]; e < e1; ++e) {
        const int64_t sidx = near_col[e];
        const T *L = Ld + 9 * e;
        const T l0 = L[0], l1 = L[1], l2 = L[2], l3 = L[3], l4 = L[4], l5 = L[5], l6 = L[6], l7 = L[7], l8 = L[8];
        const C<T> *c = cT + sidx * 3 * R;
#pragma unroll
        for (int j = 0; j < RB; ++j) {
            const int32_t r = r0 + 32 * j;
            if (r < R) {
                const C<T> c0 = c[r], c1 = c[R + r], c2 = c[2 * R + r];
                acc[0][j].x += l0 * c0.x + l1 * c1.x + l2 * c2.x;
                acc[0][j].y += l0 * c0.y + l1 * c1.y + l2 * c2.y;
                acc[1][j].x += l3 * c0.x + l4 * c1.x + l5 * c2.x;
                acc[1][j].y += l3 * c0.y + l4 * c1.y + l5 * c2.y;
                acc[2][j].x += l6 * c0.x + l7 * c1.x + l8 * c2.x;
                acc[2][j].y += l6 * c0.y + l7 * c1.y + l8 * c2.y;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < RB; ++j) {
        const int32_t r = r0 + 32 * j;
        if (r < R)
#pragma unroll
            for (int k = 0; k < 3; ++k) ynear[(t * 3 + k) * R + r] = acc[k][j];
    }
}

// J_q[c] = sum_k c_T[k] (w_q/2)(r_q - v_k)_c for every sample point.
template <typename T>
__global__ void k_point_currents(const C<T> *__restrict__ c_tri, const T *__restrict__ mom, int64_t nt, int Q,
                                 int32_t nrhs, C<T> *__restrict__ jq) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t npt = nt * Q;
    if (i >= npt * nrhs) return;
    int64_t r = i / npt, pt = i % npt, t = pt / Q;
    const C<T> *c = c_tri + (r * nt + t) * 3;
    C<T> c0 = c[0], c1 = c[1], c2 = c[2];
    const T *m = mom + 9 * pt;
    for (int d = 0; d < 3; ++d) {
        C<T> j = cscale(c0, m[d]);
        j = cadd(j, cscale(c1, m[3 + d]));
        j = cadd(j, cscale(c2, m[6 + d]));
        jq[i * 3 + d] = j;
    }
}

// Q_g[c][n] = sum over the points whose stencil holds node n of L_n(r_q) J_q[c].
// One thread per (node, group of up to 4 right-hand sides): each gather-list
// entry (point, weight) is read once for the group.
template <typename T>
__global__ void k_project(const C<T> *__restrict__ jq, int64_t npt, const int64_t *__restrict__ ptr,
                          const int32_t *__restrict__ pt, const T *__restrict__ w, int64_t Ng, int32_t nrhs,
                          C<T> *__restrict__ grid) {
    constexpr int RG = 4;
    const int32_t ngroups = (nrhs + RG - 1) / RG;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= Ng * ngroups) return;
    const int64_t g = i / Ng, n = i % Ng;
    const int32_t r0 = int32_t(g) * RG;
    const int nr = min(RG, nrhs - r0);
    C<T> a[RG][3];
#pragma unroll
    for (int k = 0; k < RG; ++k) a[k][0] = a[k][1] = a[k][2] = mk<T>(0, 0);
    const int64_t e1 = ptr[n + 1];
    for (int64_t e = ptr[n]; e < e1; ++e) {
        const int64_t p3 = int64_t(pt[e]) * 3;
        const T we = w[e];
#pragma unroll
        for (int k = 0; k < RG; ++k) {
            if (k < nr) {
                const C<T> *j = jq + (int64_t(r0 + k) * npt) * 3 + p3;
                a[k][0] = cadd(a[k][0], cscale(j[0], we));
                a[k][1] = cadd(a[k][1], cscale(j[1], we));
                a[k][2] = cadd(a[k][2], cscale(j[2], we));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < RG; ++k) {
        if (k < nr) {
            C<T> *gr = grid + int64_t(r0 + k) * 3 * Ng;
            gr[n] = a[k][0];
            gr[Ng + n] = a[k][1];
            gr[2 * Ng + n] = a[k][2];
        }
    }
}

// Phi_q[c] = sum_{n in S(q)} L_n(r_q) phi_g[c][n].
template <typename T>
__global__ void k_point_potentials(const C<T> *__restrict__ grid, const int32_t *__restrict__ start,
                                   const T *__restrict__ lw, int O, int Ny, int Nz, int64_t Ng, int64_t npt,
                                   int32_t nrhs, C<T> *__restrict__ phiq) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= npt * nrhs) return;
    int64_t r = i / npt, pt = i % npt;
    const int sx = start[3 * pt], sy = start[3 * pt + 1], sz = start[3 * pt + 2];
    const T *wx = lw + (3 * pt) * O, *wy = wx + O, *wz = wy + O;
    const C<T> *g = grid + r * 3 * Ng;
    C<T> a[3] = {mk<T>(0, 0), mk<T>(0, 0), mk<T>(0, 0)};
    for (int ii = 0; ii < O; ++ii)
        for (int jj = 0; jj < O; ++jj) {
            T wxy = wx[ii] * wy[jj];
            int64_t rowb = (int64_t(sx + ii) * Ny + (sy + jj)) * Nz + sz;
            for (int kk = 0; kk < O; ++kk) {
                T wgt = wxy * wz[kk];
                for (int c = 0; c < 3; ++c) a[c] = cadd(a[c], cscale(g[c * Ng + rowb + kk], wgt));
            }
        }
    for (int c = 0; c < 3; ++c) phiq[i * 3 + c] = a[c];
}

// Per triangle and right-hand side: far (interpolated), near (pre-corrected)
// and Gram terms combined into y_T[k] (FP64).
template <typename T>
__global__ void k_tri_out(const C<T> *__restrict__ phiq, const T *__restrict__ mom, const C<T> *__restrict__ c_tri,
                          const int64_t *__restrict__ near_ptr, const int32_t *__restrict__ near_col,
                          const T *__restrict__ Ld, const C<T> *__restrict__ ynear, const double *__restrict__ gram,
                          const int32_t *__restrict__ cond, const double *__restrict__ coef, int ncond, int64_t nt,
                          int Q, int32_t nrhs, double2 *__restrict__ y_tri) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nt * nrhs) return;
    int64_t r = i / nt, t = i % nt;
    // far: sum_q mom_q[k] . Phi_q
    C<T> far[3] = {mk<T>(0, 0), mk<T>(0, 0), mk<T>(0, 0)};
    for (int q = 0; q < Q; ++q) {
        const int64_t pt = t * Q + q;
        const C<T> *ph = phiq + (r * nt * Q + pt) * 3;
        C<T> p0 = ph[0], p1 = ph[1], p2 = ph[2];
        const T *m = mom + 9 * pt;
        for (int k = 0; k < 3; ++k) {
            far[k] = cadd(far[k], cscale(p0, m[3 * k]));
            far[k] = cadd(far[k], cscale(p1, m[3 * k + 1]));
            far[k] = cadd(far[k], cscale(p2, m[3 * k + 2]));
        }
    }
    // near: sum_T' L_d(T, T') c_T'
    C<T> nr[3] = {mk<T>(0, 0), mk<T>(0, 0), mk<T>(0, 0)};
    const C<T> *cr = c_tri + r * nt * 3;
    if (ynear) {
        for (int k = 0; k < 3; ++k) nr[k] = ynear[(t * 3 + k) * nrhs + r];
    } else for (int64_t e = near_ptr[t]; e < near_ptr[t + 1]; ++e) {
        const C<T> *c = cr + int64_t(near_col[e]) * 3;
        C<T> c0 = c[0], c1 = c[1], c2 = c[2];
        const T *L = Ld + 9 * e;
        for (int k = 0; k < 3; ++k) {
            nr[k] = cadd(nr[k], cscale(c0, L[3 * k]));
            nr[k] = cadd(nr[k], cscale(c1, L[3 * k + 1]));
            nr[k] = cadd(nr[k], cscale(c2, L[3 * k + 2]));
        }
    }
    const C<T> *ct = cr + t * 3;
    const double *gm = gram + 9 * t;
    const double *cf = coef + r * (2 * ncond + 1);
    const int cd = cond[t];
    const double zr = cf[2 * cd], zi = cf[2 * cd + 1], cl = cf[2 * ncond];
    for (int k = 0; k < 3; ++k) {
        double gr = 0.0, gi = 0.0;
        for (int l = 0; l < 3; ++l) { gr += gm[3 * k + l] * double(ct[l].x); gi += gm[3 * k + l] * double(ct[l].y); }
        double fr = double(far[k].x) + double(nr[k].x), fi = double(far[k].y) + double(nr[k].y);
        // Z_s * gram + j c_L * (far + near)
        double yr = zr * gr - zi * gi - cl * fi;
        double yi = zr * gi + zi * gr + cl * fr;
        y_tri[i * 3 + k] = make_double2(yr, yi);
    }
}

// y_b = sum over the branch's two triangles of s * y_T[k].
__global__ void k_branch_out(const double2 *__restrict__ y_tri, const int32_t *__restrict__ br_tri,
                             const int8_t *__restrict__ br_local, int64_t nt, int64_t nb, int64_t ldy, int32_t nrhs,
                             double2 *__restrict__ y) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= ldy * nrhs) return;
    int64_t r = i / ldy, b = i % ldy;
    double2 v = make_double2(0.0, 0.0);
    if (b < nb) {
        double2 a = y_tri[(r * nt + br_tri[2 * b]) * 3 + br_local[2 * b]];
        double2 c = y_tri[(r * nt + br_tri[2 * b + 1]) * 3 + br_local[2 * b + 1]];
        v = csub(a, c);
    }
    y[i] = v;
}

// Tour values for A: +delta(v) at v's enter slot, -delta(v) at its exit slot,
// delta(v) = voltage of v's parent twig walked from v towards the root.
__global__ void k_tour_voltage(const double2 *__restrict__ y_br, int64_t ldy, double2 *__restrict__ tour,
                               int64_t nslots, const int32_t *__restrict__ tour_node,
                               const int8_t *__restrict__ tour_enter, const int32_t *__restrict__ parent_branch,
                               const int32_t *__restrict__ tail, int32_t nrhs) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nslots * nrhs) return;
    int64_t r = i / nslots, s = i % nslots;
    int v = tour_node[s];
    int t = parent_branch[v];
    double2 d = make_double2(0.0, 0.0);
    if (t >= 0) {
        d = y_br[r * ldy + t];
        if (tail[t] != v) { d.x = -d.x; d.y = -d.y; }
        if (!tour_enter[s]) { d.x = -d.x; d.y = -d.y; }
    }
    tour[i] = d;
}

__global__ void k_loop_out(const double2 *__restrict__ y_br, int64_t ldy, const double2 *__restrict__ P,
                           int64_t nslots, const int32_t *__restrict__ link_branch, const int32_t *__restrict__ tail,
                           const int32_t *__restrict__ head, const int32_t *__restrict__ enter, int64_t nl,
                           int32_t nrhs, double2 *__restrict__ y) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nl * nrhs) return;
    int64_t r = i / nl, l = i % nl;
    int32_t e = link_branch[l];
    const double2 *row = P + r * nslots;
    double2 v = y_br[r * ldy + e];
    v = cadd(v, row[enter[head[e]]]);
    v = csub(v, row[enter[tail[e]]]);
    y[i] = v;
}

inline unsigned nblk(int64_t n, int t = 256) { return unsigned((n + t - 1) / t); }

}  // namespace

namespace sie {

int scratch_reserve(pfft_plan *p, int32_t nrhs, int prec) {
    Scratch &s = p->scr;
    if (s.cap_rhs >= nrhs && s.prec == prec) return SIE_OK;
    for (void *a : {s.tour, s.c_tri, s.jq, s.grid, s.spec, s.y_tri, s.y_br, (void *)s.coef, s.cT, s.ynear})
        if (a) cudaFree(a);
    s = Scratch{};
    const size_t cs = prec == SIE_PREC_FP64 ? sizeof(double2) : sizeof(float2);
    const int64_t R = std::max<int32_t>(nrhs, 1);
    const size_t sizes[10] = {
        size_t(R) * 2 * p->nn * sizeof(double2),
        size_t(R) * p->nt * 3 * cs,
        size_t(R) * p->nt * p->Q * 3 * cs,
        size_t(R) * 3 * p->Ng * cs,
        size_t(R) * 3 * p->Nx * p->My * p->Mz * cs,
        size_t(R) * p->nt * 3 * sizeof(double2),
        size_t(R) * (p->nb + p->np) * sizeof(double2),
        size_t(R) * (2 * p->ncond + 1) * sizeof(double),
        size_t(R) * p->nt * 3 * cs,
        size_t(R) * p->nt * 3 * cs};
    void **dst[10] = {&s.tour, &s.c_tri, &s.jq, &s.grid, &s.spec, &s.y_tri, &s.y_br, (void **)&s.coef, &s.cT, &s.ynear};
    for (int i = 0; i < 10; ++i) {
        cudaError_t e = cudaMalloc(dst[i], std::max<size_t>(sizes[i], 16));
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) { cudaFree(*dst[j]); *dst[j] = nullptr; }
            set_error(std::string("scratch allocation failed: ") + cudaGetErrorString(e));
            s = Scratch{};
            return SIE_ERR_OOM;
        }
        s.bytes += sizes[i];
    }
    s.phiq = s.jq;   // the point currents are consumed before the potentials are written
    s.cap_rhs = int32_t(R);
    s.prec = prec;
    return SIE_OK;
}

template <typename T>
int matvec_t(pfft_plan *p, const double2 *x, double2 *y, int32_t R, int space, cudaStream_t st) {
    Scratch &s = p->scr;
    const int64_t nslots = 2 * p->nn;
    const int64_t ldy = p->nb + p->np;
    double2 *tour = (double2 *)s.tour;
    C<T> *c_tri = (C<T> *)s.c_tri, *jq = (C<T> *)s.jq, *grid = (C<T> *)s.grid, *spec = (C<T> *)s.spec;
    double2 *y_tri = (double2 *)s.y_tri, *y_br = (double2 *)s.y_br;
    const T *mom, *lw, *pjw, *Ld;
    if constexpr (sizeof(T) == 8) {
        mom = (const T *)p->d_mom64; lw = (const T *)p->d_lw64; pjw = (const T *)p->d_pj_w64; Ld = (const T *)p->d_Ld64;
    } else {
        mom = (const T *)p->d_mom32; lw = (const T *)p->d_lw32; pjw = (const T *)p->d_pj_w32; Ld = (const T *)p->d_Ld32;
    }
    std::unique_ptr<StageTimer> tm(new StageTimer(p, SIE_STAGE_LOOP_TO_BRANCH, st));
    if (space == SIE_SPACE_LOOP) {
        k_tour_inject<<<nblk(nslots * R), 256, 0, st>>>(x, p->nl, tour, nslots, p->d_tour_node, p->d_tour_enter,
                                                         p->d_nl_ptr, p->d_nl_loop, p->d_nl_sign, R);
        SIE_LAUNCH_CHECK(p);
        k_scan_rows<<<R, 1024, 0, st>>>(tour, nslots);
        SIE_LAUNCH_CHECK(p);
    }
    k_alpha_tri<T><<<nblk(p->nt * 3 * R), 256, 0, st>>>(x, p->nl, tour, nslots, p->d_tb, p->d_ts, p->d_loop_of_branch,
                                                         p->d_twig_node, p->d_head, p->d_enter, p->d_exit, p->nt, R,
                                                         space, p->nb, c_tri, (C<T> *)s.cT);
    SIE_LAUNCH_CHECK(p);
    const int64_t npt = p->nt * p->Q;
    tm.reset(new StageTimer(p, SIE_STAGE_POINT_CURRENTS, st));
    k_point_currents<T><<<nblk(npt * R), 256, 0, st>>>(c_tri, mom, p->nt, p->Q, R, jq);
    SIE_LAUNCH_CHECK(p);
    tm.reset(new StageTimer(p, SIE_STAGE_PROJECT, st));
    k_project<T><<<nblk(p->Ng * ((R + 3) / 4)), 256, 0, st>>>(jq, npt, p->d_pj_ptr, p->d_pj_pt, pjw, p->Ng, R, grid);
    SIE_LAUNCH_CHECK(p);
    tm.reset();
    int rc = fft_conv(p, grid, spec, R, sizeof(T) == 8 ? SIE_PREC_FP64 : SIE_PREC_MIXED, st);
    if (rc) return rc;
    C<T> *phiq = (C<T> *)s.phiq;
    tm.reset(new StageTimer(p, SIE_STAGE_INTERP, st));
    k_point_potentials<T><<<nblk(npt * R), 256, 0, st>>>(grid, p->d_start, lw, p->O, p->Ny, p->Nz, p->Ng, npt, R, phiq);
    SIE_LAUNCH_CHECK(p);
    C<T> *ynear = nullptr;
    if (R >= 16) {   // batched right-hand sides: near field as a block-sparse x dense product
        tm.reset(new StageTimer(p, SIE_STAGE_NEAR, st));
        ynear = (C<T> *)s.ynear;
        const int32_t nchunk = (R + 127) / 128;
        const int64_t warps = p->nt * nchunk;
        k_near_spmm<T, 4><<<nblk(warps * 32, 256), 256, 0, st>>>(p->d_near_ptr, p->d_near_col, Ld, (const C<T> *)s.cT,
                                                                p->nt, R, nchunk, ynear);
        SIE_LAUNCH_CHECK(p);
        tm.reset(new StageTimer(p, SIE_STAGE_INTERP, st));
    }
    k_tri_out<T><<<nblk(p->nt * R, 128), 128, 0, st>>>(phiq, mom, c_tri, p->d_near_ptr, p->d_near_col, Ld, ynear,
                                                   p->d_gram, p->d_cond, s.coef, p->ncond, p->nt, p->Q, R, y_tri);
    SIE_LAUNCH_CHECK(p);
    tm.reset(new StageTimer(p, SIE_STAGE_BRANCH_TO_LOOP, st));
    if (space == SIE_SPACE_BRANCH) {
        k_branch_out<<<nblk(p->nb * R), 256, 0, st>>>(y_tri, p->d_br_tri, p->d_br_local, p->nt, p->nb, p->nb, R, y);
        SIE_LAUNCH_CHECK(p);
        return SIE_OK;
    }
    k_branch_out<<<nblk(ldy * R), 256, 0, st>>>(y_tri, p->d_br_tri, p->d_br_local, p->nt, p->nb, ldy, R, y_br);
    SIE_LAUNCH_CHECK(p);
    k_tour_voltage<<<nblk(nslots * R), 256, 0, st>>>(y_br, ldy, tour, nslots, p->d_tour_node, p->d_tour_enter,
                                                      p->d_parent_branch, p->d_tail, R);
    SIE_LAUNCH_CHECK(p);
    k_scan_rows<<<R, 1024, 0, st>>>(tour, nslots);
    SIE_LAUNCH_CHECK(p);
    k_loop_out<<<nblk(p->nl * R), 256, 0, st>>>(y_br, ldy, tour, nslots, p->d_link_branch, p->d_tail, p->d_head,
                                                 p->d_enter, p->nl, R, y);
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

// Per right-hand side: Z_s of each conductor and c_L / j (Eq. ImpedanceOp, Eq. Zb).
int upload_coef(pfft_plan *p, const double *omega, int32_t R, cudaStream_t st) {
    std::vector<double> cf(size_t(R) * (2 * p->ncond + 1));
    for (int32_t r = 0; r < R; ++r) {
        const double w = omega[r];
        if (!(w >= 0.0) || !std::isfinite(w)) return fail(SIE_ERR_ARG, "pfft_matvec: omega must be finite and >= 0");
        for (int c = 0; c < p->ncond; ++c) {
            double zs = std::sqrt(w * kMu0 / (2.0 * p->sigma[c]));
            cf[r * (2 * p->ncond + 1) + 2 * c] = zs;
            cf[r * (2 * p->ncond + 1) + 2 * c + 1] = zs;
        }
        cf[r * (2 * p->ncond + 1) + 2 * p->ncond] = w * kMu0 / (4.0 * M_PI);
    }
    SIE_CUDA(cudaMemcpyAsync(p->scr.coef, cf.data(), cf.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    return SIE_OK;
}

int matvec_async(pfft_plan *p, const void *x, void *y, int32_t nrhs, const double *omega, int space, int prec,
                 cudaStream_t st) {
    int rc = scratch_reserve(p, nrhs, prec);
    if (rc) return rc;
    rc = upload_coef(p, omega, nrhs, st);
    if (rc) return rc;
    if (prec == SIE_PREC_FP64)
        return matvec_t<double>(p, (const double2 *)x, (double2 *)y, nrhs, space, st);
    return matvec_t<float>(p, (const double2 *)x, (double2 *)y, nrhs, space, st);
}

}  // namespace sie

extern "C" int pfft_matvec(pfft_plan *p, const void *x, void *y, int32_t nrhs, const double *omega, int32_t space,
                           int32_t prec, void *cuda_stream) {
    if (!p || !x || !y || !omega) return fail(SIE_ERR_ARG, "pfft_matvec: NULL argument");
    if (nrhs < 1) return fail(SIE_ERR_ARG, "pfft_matvec: nrhs must be >= 1");
    if (space != SIE_SPACE_LOOP && space != SIE_SPACE_BRANCH) return fail(SIE_ERR_ARG, "pfft_matvec: bad space");
    if (prec != SIE_PREC_FP64 && prec != SIE_PREC_MIXED) return fail(SIE_ERR_ARG, "pfft_matvec: bad precision");
    const int64_t n = space == SIE_SPACE_LOOP ? p->nl : p->nb;
    const char *xb = (const char *)x, *yb = (const char *)y;
    const size_t bytes = size_t(nrhs) * n * sizeof(double2);
    if (xb < yb + bytes && yb < xb + bytes) return fail(SIE_ERR_ARG, "pfft_matvec: x and y overlap");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    (void)cudaGetLastError();   // clear a stale error left by earlier work in this thread
    int rc = sie::matvec_async(p, x, y, nrhs, omega, space, prec, st);
    if (rc) return rc;
    SIE_CUDA(cudaStreamSynchronize(st));
    return SIE_OK;
}
