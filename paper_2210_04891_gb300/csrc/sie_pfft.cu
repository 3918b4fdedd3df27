// pfft_matvec: the loop-space product of Eq. (FinalME) with the inductive part
// applied by the pre-corrected FFT (Sec. IV-A, IV-B of arXiv 2210.04891):
//
//   alpha = A^T x                     (Eq. CurT; Euler-tour subtree sums)
//   Q_g   = sum_T W(n,T) c_T          (Eq. Projection with the point currents
//                                      J_q = sum_k c_k (w_q/2)(r_q - v_k) folded in)
//   phi_g = H Q_g                     (Eq. FFTCal; zero-padded FFT convolution)
//   y_T   = Z_s G_T c_T + c_L (sum_n W(n,T)^T phi_n + sum_T' L_d(T,T') c_T')
//                                     (Eq. interpolation with I = B^T, Eq. Zb, Eq. Lb)
//   y     = A y_b                     (Eq. VolT; Euler-tour root-path sums)
//
// A^T x: the current of a twig equals minus the current its subtree receives
// through links (Kirchhoff's current law), a subtree sum = a difference of two
// prefix sums along the Euler tour.  A y: the voltage of a fundamental loop is
// its link's voltage plus psi(head) - psi(tail), psi(v) the sum of twig
// voltages on v's path to the root = a prefix sum of +-delta over the tour.
// Both are exact rewrites of the sparse products (no approximation).
//
// Projection, interpolation and near field are block-sparse x dense products
// with 3x3 real blocks and complex right-hand sides: every dense operand is
// stored with the right-hand sides innermost (c_T as [T][3][R], potentials as
// [n][3][R]), one warp reads a block once and applies it to a slab of up to
// 128 right-hand sides with coalesced loads.
#include <algorithm>
#include <cmath>
#include <complex>
#include <memory>
#include <type_traits>
#include <vector>

#include "sie_dd.cuh"
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

// Elements of the loop/branch maps after the field computation: complex128 in
// the FP64 form, double-float float4 (sie_dd.cuh) in the mixed and double-float forms.
template <typename T> using TourE = typename std::conditional<std::is_same<T, double>::value, double2, float4>::type;
template <typename T> constexpr bool is_f32 = std::is_same<T, float>::value;
template <typename T> constexpr bool is_f64 = std::is_same<T, double>::value;
template <typename T> constexpr bool is_df = std::is_same<T, df>::value;

__device__ __forceinline__ double2 eadd(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ float4 eadd(float4 a, float4 b) {
    return cdd(dd_add(cdd_re(a), cdd_re(b)), dd_add(cdd_im(a), cdd_im(b)));
}
__device__ __forceinline__ double2 eneg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ float4 eneg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
template <typename E> __device__ __forceinline__ E ezero();
template <> __device__ __forceinline__ double2 ezero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float4 ezero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
// conversions: FP64 value -> element; element -> FP64, FP32 or another element type
__device__ __forceinline__ void eset(double2 &e, double2 v) { e = v; }
__device__ __forceinline__ void eset(float4 &e, double2 v) { e = cdd(dd_from(v.x), dd_from(v.y)); }
__device__ __forceinline__ void eset(double2 &e, float4 v) {
    e = make_double2(double(v.x) + double(v.y), double(v.z) + double(v.w));
}
__device__ __forceinline__ void eset(float4 &e, float4 v) { e = v; }
__device__ __forceinline__ double2 to_c(double2 v, double2) { return v; }
__device__ __forceinline__ float2 to_c(double2 v, float2) { return make_float2(float(v.x), float(v.y)); }
__device__ __forceinline__ float2 to_c(float4 e, float2) { return make_float2(e.x + e.y, e.z + e.w); }
__device__ __forceinline__ cdf to_c(double2 v, cdf) {
    const DD a = dd_from(v.x), b = dd_from(v.y);
    return cdf{df(a.hi, a.lo), df(b.hi, b.lo)};
}
__device__ __forceinline__ cdf to_c(float4 e, cdf) { return cdf{df(e.x, e.y), df(e.z, e.w)}; }
__device__ __forceinline__ float4 shfl_up(float4 v, int d) {
    v.x = __shfl_up_sync(0xffffffffu, v.x, d);
    v.y = __shfl_up_sync(0xffffffffu, v.y, d);
    v.z = __shfl_up_sync(0xffffffffu, v.z, d);
    v.w = __shfl_up_sync(0xffffffffu, v.w, d);
    return v;
}

// Inclusive prefix sum of each row of a [R][n] array of elements, in place.
// One CTA of 1024 threads per row, 4 items per thread per chunk; the next
// chunk's loads are issued before the current chunk's block scan.
template <typename E>
__global__ void __launch_bounds__(1024) k_scan_rows(E *buf, int64_t n) {
    __shared__ E warp_tot[32];
    __shared__ E carry_s;
    E *row = buf + blockIdx.x * n;
    E carry = ezero<E>();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    E vn[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = 4 * int64_t(threadIdx.x) + k;
        vn[k] = i < n ? row[i] : ezero<E>();
    }
    for (int64_t base = 0; base < n; base += 4 * 1024) {
        E v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = vn[k];
        const int64_t i0 = base + 4 * int64_t(threadIdx.x);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = i0 + 4 * 1024 + k;
            vn[k] = i < n ? row[i] : ezero<E>();
        }
        E run = ezero<E>();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            run = eadd(run, v[k]);
            v[k] = run;
        }
        E incl = run;   // warp inclusive scan of thread totals
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            E o = shfl_up(incl, d);
            if (lane >= d) incl = eadd(incl, o);
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            E w = warp_tot[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                E o = shfl_up(w, d);
                if (lane >= d) w = eadd(w, o);
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        E off = carry;
        if (warp > 0) off = eadd(off, warp_tot[warp - 1]);
        off = eadd(off, eadd(incl, eneg(run)));   // exclusive within the warp
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k < n) row[i0 + k] = eadd(v[k], off);
        if (threadIdx.x == 1023) carry_s = eadd(off, run);
        __syncthreads();
        carry = carry_s;
        __syncthreads();
    }
}

// Tour values for A^T: at node v's enter slot the current the links inject
// into v (+x on links entering v, -x on links leaving it); 0 at exit slots.
// Grid (slots, right-hand-side groups): a thread takes one slot and kTourRc
// right-hand sides, so the slot's index chain (node, link list, loops) is read
// once for the group and the group's loads of x are independent.
constexpr int kTourRc = 8;
template <typename E>
__global__ void k_tour_inject(const double2 *__restrict__ x, int64_t nl, E *__restrict__ tour, int64_t nslots,
                              const int32_t *__restrict__ tour_node, const int8_t *__restrict__ tour_enter,
                              const int32_t *__restrict__ nl_ptr, const int32_t *__restrict__ nl_loop,
                              const int8_t *__restrict__ nl_sign, int32_t nrhs) {
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    const int32_t r0 = int32_t(blockIdx.y) * kTourRc;
    const int nr = min(kTourRc, nrhs - r0);
    const int v = tour_node[s];
    int32_t k0 = 0, k1 = 0;
    if (tour_enter[s]) {
        k0 = nl_ptr[v];
        k1 = nl_ptr[v + 1];
    }
    if (k1 <= k0) {   // no link at this slot (most slots): zeros, no FP64 work
#pragma unroll
        for (int j = 0; j < kTourRc; ++j)
            if (j < nr) tour[int64_t(r0 + j) * nslots + s] = ezero<E>();
        return;
    }
    double2 acc[kTourRc];   // a few link currents, exact inputs
#pragma unroll
    for (int j = 0; j < kTourRc; ++j) acc[j] = make_double2(0.0, 0.0);
    for (int32_t k = k0; k < k1; ++k) {
        const double2 *xl = x + int64_t(r0) * nl + nl_loop[k];
        const bool pos = nl_sign[k] > 0;
#pragma unroll
        for (int j = 0; j < kTourRc; ++j)
            if (j < nr) {
                const double2 xv = xl[int64_t(j) * nl];
                acc[j] = pos ? cadd(acc[j], xv) : csub(acc[j], xv);
            }
    }
    // the conversion to the tour's element (double-float pairs in the mixed
    // form) runs on the FP64 pipe: only here, on the slots that carry links
#pragma unroll
    for (int j = 0; j < kTourRc; ++j)
        if (j < nr) {
            E out;
            eset(out, acc[j]);
            tour[int64_t(r0 + j) * nslots + s] = out;
        }
}

// Branch current of branch b for right-hand side r (loop space): a link carries
// its loop current; a twig above node v carries -sigma * (subtree inflow), a
// difference of two prefix sums taken in the tour's arithmetic.
template <typename T, typename E>
__device__ __forceinline__ C<T> branch_current(int32_t b, int64_t r, const double2 *__restrict__ x, int64_t nl,
                                               const E *__restrict__ P, int64_t nslots,
                                               const int32_t *__restrict__ loop_of_branch,
                                               const int32_t *__restrict__ twig_node, const int32_t *__restrict__ head,
                                               const int32_t *__restrict__ enter, const int32_t *__restrict__ exit_) {
    int32_t l = loop_of_branch[b];
    if (l >= 0) return to_c(x[r * nl + l], C<T>{});
    int32_t v = twig_node[b];
    const E *row = P + r * nslots;
    E S = row[exit_[v]];
    int32_t e = enter[v];
    if (e > 0) S = eadd(S, eneg(row[e - 1]));
    const C<T> d = to_c(S, C<T>{});
    return head[b] == v ? mk<T>(-d.x, -d.y) : d;
}

// Local currents c_T[k] = s_k alpha_{b(T,k)}: one thread per (T, r) for the
// three local edges, written as cT [T][3][R] (right-hand sides innermost).
template <typename T>
__global__ void k_alpha_tri(const double2 *__restrict__ x, int64_t nl, const TourE<T> *__restrict__ P, int64_t nslots,
                            const int32_t *__restrict__ tb, const int8_t *__restrict__ ts,
                            const int32_t *__restrict__ loop_of_branch, const int32_t *__restrict__ twig_node,
                            const int32_t *__restrict__ head, const int32_t *__restrict__ enter,
                            const int32_t *__restrict__ exit_, int64_t nt, int32_t nrhs, int space, int64_t nb,
                            C<T> *__restrict__ cT) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nt * nrhs) return;
    const int64_t t = i / nrhs, r = i % nrhs;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t tk = t * 3 + k;
        const int32_t b = tb[tk];
        C<T> a = mk<T>(T(0), T(0));
        if (b >= 0) {
            if (space == SIE_SPACE_LOOP)
                a = branch_current<T>(b, r, x, nl, P, nslots, loop_of_branch, twig_node, head, enter, exit_);
            else
                a = to_c(x[r * nb + b], C<T>{});
            if (ts[tk] < 0) { a.x = -a.x; a.y = -a.y; }
        }
        cT[tk * nrhs + r] = a;
    }
}

// acc += b x for double-float b and x into an unnormalised double-float sum:
// the high part takes one FP32 add per term (the chain a gather runs along),
// the two-product error of the high parts, the two-sum error of that add and
// the cross products of high and low parts go to the low part, one add per
// term.  A sum of n terms keeps about 48 bits plus log2(n); readers treat
// (hi, lo) as the value hi + lo, whatever its normalisation.
__device__ __forceinline__ void df_acc(df &acc, df b, df x) {
    const float p = b.hi * x.hi;
    const float e = fmaf(b.hi, x.hi, -p);
    const float s = acc.hi + p, bb = s - acc.hi;
    const float f = (acc.hi - (s - bb)) + (p - bb);
    acc.hi = s;
    acc.lo += fmaf(b.lo, x.hi, fmaf(b.hi, x.lo, e + f));
}
// the same value as a normalised pair (two-sum of its parts)
__device__ __forceinline__ df df_norm(df a) {
    const float s = a.hi + a.lo, bb = s - a.hi;
    return df(s, (a.hi - (s - bb)) + (a.lo - bb));
}

// V complex values at p (16-byte aligned when V = 2).
template <typename T, int V> __device__ __forceinline__ void ldv(const C<T> *p, C<T> (&v)[V]) {
    if constexpr (V == 2) {
        static_assert(is_f32<T>, "two complex per load only in FP32");
        const float4 u = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = make_float2(u.x, u.y);
        v[1] = make_float2(u.z, u.w);
    } else if constexpr (is_df<T>) {
        const float4 u = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = cdf{df(u.x, u.y), df(u.z, u.w)};
    } else {
        v[0] = __ldg(p);
    }
}
template <typename T, int V> __device__ __forceinline__ void stv(C<T> *p, const C<T> (&v)[V]) {
    if constexpr (is_df<T>) {
        *p = cdf{df_norm(v[0].x), df_norm(v[0].y)};
    } else if constexpr (V == 2) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    } else {
        *p = v[0];
    }
}

// acc[a][j][v] += sum over the records e of row [e0, e1) of
//                 sum_b rec_e.b[3a+b] X[col_e][b][r],   r = rl + 32 V j + v.
// X is [rows][3][R] (right-hand sides innermost).  FULL: every r < R.
// UNR records in flight per warp (measured: 1 for the projection, 4 for the
// interpolation and the triangle gathers).
template <typename T, int V, int J, bool FULL, int UNR = 4>
__device__ __forceinline__ void gather_rows(const Rec<T> *__restrict__ rec, int64_t e0, int64_t e1,
                                            const C<T> *__restrict__ X, int32_t R, int32_t rl,
                                            C<T> (&acc)[3][J][V]) {
    const int64_t ld = 3 * int64_t(R);
#pragma unroll UNR
    for (int64_t e = e0; e < e1; ++e) {
        T b[9];
        const int64_t col = load_rec<T>(rec + e, b);
        const C<T> *x = X + col * ld;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int32_t r = rl + 32 * V * j;
            if (FULL || r < R) {
                C<T> x0[V], x1[V], x2[V];
                ldv<T, V>(x + r, x0);
                ldv<T, V>(x + R + r, x1);
                ldv<T, V>(x + 2 * R + r, x2);
#pragma unroll
                for (int v = 0; v < V; ++v)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if constexpr (is_df<T>) {
                            df_acc(acc[a][j][v].x, b[3 * a], x0[v].x);
                            df_acc(acc[a][j][v].x, b[3 * a + 1], x1[v].x);
                            df_acc(acc[a][j][v].x, b[3 * a + 2], x2[v].x);
                            df_acc(acc[a][j][v].y, b[3 * a], x0[v].y);
                            df_acc(acc[a][j][v].y, b[3 * a + 1], x1[v].y);
                            df_acc(acc[a][j][v].y, b[3 * a + 2], x2[v].y);
                        } else {
                            acc[a][j][v].x += b[3 * a] * x0[v].x + b[3 * a + 1] * x1[v].x + b[3 * a + 2] * x2[v].x;
                            acc[a][j][v].y += b[3 * a] * x0[v].y + b[3 * a + 1] * x1[v].y + b[3 * a + 2] * x2[v].y;
                        }
                    }
            }
        }
    }
}

template <typename T, int V, int J> __device__ __forceinline__ void zero(C<T> (&acc)[3][J][V]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[a][j][v] = mk<T>(T(0), T(0));
}

// Grid currents (Eq. Projection): Q_g[d][n] = sum_T sum_k W(n,T)[d][k] c_T[k]
// for a slab of 32 V J right-hand sides.  A block of 8 warps takes 8
// consecutive nodes, one per warp (lanes over right-hand sides); the block's
// results go through shared memory so that each of the 3 x slab grids gets an
// 8-node run per block.  Grid layout [3][R][Ng].
constexpr int kProjNodes = 8;
template <typename T, int V, int J> __host__ __device__ constexpr int proj_rows() { return 3 * 32 * V * J + 2; }
template <typename T, int V, int J> constexpr size_t proj_smem() {
    return size_t(kProjNodes) * proj_rows<T, V, J>() * sizeof(C<T>);
}

template <typename T, int V, int J>
__global__ void __launch_bounds__(256) k_project(const int64_t *__restrict__ ptr, const Rec<T> *__restrict__ rec,
                                                 const C<T> *__restrict__ cT, int64_t Ng, int32_t R,
                                                 C<T> *__restrict__ grid) {
    constexpr int SLAB = 32 * V * J;
    // row stride 3 SLAB + 2 (= 2 mod 16 complex): the 8-node reads below hit distinct banks
    constexpr int ROWS = proj_rows<T, V, J>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T> *sm = reinterpret_cast<C<T> *>(smem_raw);   // [kProjNodes][ROWS]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n0 = int64_t(blockIdx.x) * kProjNodes, n = n0 + w;
    const int32_t rbase = int32_t(blockIdx.y) * SLAB;
    const int32_t rl = rbase + V * lane;
    C<T> acc[3][J][V];
    zero<T, V, J>(acc);
    if (n < Ng) {
        if (rbase + SLAB <= R) gather_rows<T, V, J, true, 1>(rec, ptr[n], ptr[n + 1], cT, R, rl, acc);
        else gather_rows<T, V, J, false, 1>(rec, ptr[n], ptr[n + 1], cT, R, rl, acc);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int j = 0; j < J; ++j) stv<T, V>(sm + w * ROWS + d * SLAB + V * lane + 32 * V * j, acc[d][j]);
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * SLAB * kProjNodes; i += blockDim.x) {
        const int row = i / kProjNodes, nd = i % kProjNodes;
        const int d = row / SLAB;
        const int32_t r = rbase + row % SLAB;
        const int64_t nn = n0 + nd;
        if (r < R && nn < Ng) grid[(int64_t(d) * R + r) * Ng + nn] = sm[nd * ROWS + row];
    }
}

// Grid currents (Eq. Projection) of the mixed form by node chunks whose
// triangles' local currents are staged in shared memory: one CTA per (chunk,
// slab of kChunkRhs right-hand sides).  The rows c_T [T][3][R] of the chunk's
// triangles are read once per slab (coalesced 256-byte rows) instead of once
// per (node, triangle) record, which the direct form reads through L2 (a
// triangle has about 57 stencil nodes); each warp then takes one node at a
// time, lanes over right-hand sides, sums its records in order (the sums of
// k_project) from the staged rows named by the records' chunk-local indices,
// and groups of 8 nodes pass through shared memory so that each grid row
// [d][r] gets runs of consecutive nodes (a tile's z extent is 8).
constexpr int kPTRows = 3 * kChunkRhs + 2;   // staging pitch: the 8-node reads hit distinct banks
constexpr size_t kPTSmem = size_t(kChunkTri) * 3 * kChunkRhs * sizeof(float2) + size_t(8) * kPTRows * sizeof(float2);

__global__ void __launch_bounds__(256, 4)
    k_project_tiled(const int32_t *__restrict__ node_ptr, const int32_t *__restrict__ nodes,
                    const int32_t *__restrict__ tri_ptr, const int32_t *__restrict__ tri,
                    const int64_t *__restrict__ pn_ptr, const Rec<float> *__restrict__ rec,
                    const uint16_t *__restrict__ lcol, const float2 *__restrict__ cT, int64_t Ng, int32_t R,
                    float2 *__restrict__ grid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *X = reinterpret_cast<float2 *>(smem_raw);   // [kChunkTri][3][kChunkRhs]
    float2 *O = X + kChunkTri * 3 * kChunkRhs;         // [8][kPTRows]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c = blockIdx.x;
    const int32_t r0 = int32_t(blockIdx.y) * kChunkRhs;
    const int32_t nr = min(kChunkRhs, R - r0);
    const int32_t t0 = tri_ptr[c], nT = tri_ptr[c + 1] - t0;
    // staging by asynchronous 8-byte copies, all in flight at once (lanes beyond
    // the slab's last right-hand side copy nothing and zero-fill)
    for (int i = w; i < 3 * nT; i += 8) {
        const int32_t t = tri[t0 + i / 3];
        const int l = i - 3 * (i / 3);
        const bool in = lane < nr;
        const float2 *src = cT + (int64_t(t) * 3 + l) * R + r0 + (in ? lane : 0);
        const uint32_t dst = uint32_t(__cvta_generic_to_shared(X + i * kChunkRhs + lane));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(in ? 8 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const int32_t n0 = node_ptr[c], nN = node_ptr[c + 1] - n0;
    for (int32_t g = 0; g < nN; g += 8) {
        float2 acc[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[d] = make_float2(0.f, 0.f);
        if (g + w < nN) {
            const int64_t n = nodes[n0 + g + w];
#pragma unroll 2
            for (int64_t e = pn_ptr[n]; e < pn_ptr[n + 1]; ++e) {
                float b[9];
                load_rec<float>(rec + e, b);
                const float2 *x = X + int(__ldg(lcol + e)) * (3 * kChunkRhs) + lane;
                const float2 x0 = x[0], x1 = x[kChunkRhs], x2 = x[2 * kChunkRhs];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    acc[a].x += b[3 * a] * x0.x + b[3 * a + 1] * x1.x + b[3 * a + 2] * x2.x;
                    acc[a].y += b[3 * a] * x0.y + b[3 * a + 1] * x1.y + b[3 * a + 2] * x2.y;
                }
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) O[w * kPTRows + d * kChunkRhs + lane] = acc[d];
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * kChunkRhs * 8; i += 256) {
            const int row = i >> 3, nd = i & 7;
            const int d = row / kChunkRhs, r = row - d * kChunkRhs;
            if (r < nr && g + nd < nN)
                grid[(int64_t(d) * R + r0 + r) * Ng + nodes[n0 + g + nd]] = O[nd * kPTRows + row];
        }
        __syncthreads();
    }
}

// Grid potentials regrouped with the right-hand sides innermost:
// phiT[n][b] = grid[b][n], b = d R + r, for the 32-node tiles that hold a
// stencil node (no other node is interpolated from).
template <typename T>
__global__ void __launch_bounds__(256) k_regroup(const C<T> *__restrict__ grid, const int32_t *__restrict__ tiles,
                                                 int64_t Ng, int32_t B, C<T> *__restrict__ phiT) {
    __shared__ C<T> s[32][33];
    const int64_t n0 = int64_t(tiles[blockIdx.x]) * 32;
    const int32_t b0 = int32_t(blockIdx.y) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int i = ty; i < 32; i += 8) {
        const int32_t b = b0 + i;
        const int64_t n = n0 + tx;
        if (b < B && n < Ng) s[i][tx] = grid[int64_t(b) * Ng + n];
    }
    __syncthreads();
#pragma unroll
    for (int i = ty; i < 32; i += 8) {
        const int64_t n = n0 + i;
        const int32_t b = b0 + tx;
        if (b < B && n < Ng) phiT[n * B + b] = s[tx][i];
    }
}

// y_T[k] = Z_s sum_l G_T[k][l] c_T[l] + j c_L f_T[k] (Eq. Zb) for the right-hand
// sides rl + 32 V j + v < R of a warp's slab, f_T = acc (FP64, or double-float
// from the FP32 field in the mixed form).
template <typename T, int V, int J>
__device__ __forceinline__ void tri_epilogue(const C<T> (&acc)[3][J][V], int64_t t, int32_t rl, int32_t R,
                                             const C<T> *__restrict__ cT, const double *__restrict__ gram,
                                             const int32_t *__restrict__ cond, const double *__restrict__ coef,
                                             const float2 *__restrict__ coef_dd, int ncond, int64_t nt,
                                             TourE<T> *__restrict__ y_tri) {
    const int cd = cond[t];
    if constexpr (is_df<T>) {
        // double-float product: Gram term and Eq. Zb in double-float like the field
        DD G[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) G[i] = dd_from(__ldg(gram + 9 * t + i));
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int32_t r = rl + 32 * V * j + v;
                if (r >= R) continue;
                const float2 *cf = coef_dd + int64_t(r) * (2 * ncond + 1);
                const float2 zr = cf[2 * cd], zi = cf[2 * cd + 1], cl = cf[2 * ncond];
                cdf c[3];
#pragma unroll
                for (int l = 0; l < 3; ++l) c[l] = cT[(t * 3 + l) * R + r];
                float4 *out = y_tri + (int64_t(r) * nt + t) * 3;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    DD gr = dd_mul(G[3 * k], to_dd(c[0].x)), gi = dd_mul(G[3 * k], to_dd(c[0].y));
#pragma unroll
                    for (int l = 1; l < 3; ++l) {
                        gr = dd_add(gr, dd_mul(G[3 * k + l], to_dd(c[l].x)));
                        gi = dd_add(gi, dd_mul(G[3 * k + l], to_dd(c[l].y)));
                    }
                    out[k] = dd_zb_df(zr, zi, cl, gr, gi, to_dd(df_norm(acc[k][j][v].x)),
                                         to_dd(df_norm(acc[k][j][v].y)));
                }
            }
    } else if constexpr (is_f32<T>) {
        // mixed form: Gram term in FP32 like the field, Eq. Zb in double-float
        float G[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) G[i] = float(__ldg(gram + 9 * t + i));
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int32_t r = rl + 32 * V * j + v;
                if (r >= R) continue;
                const float2 *cf = coef_dd + int64_t(r) * (2 * ncond + 1);
                const float2 zr = cf[2 * cd], zi = cf[2 * cd + 1], cl = cf[2 * ncond];
                float2 c[3];
#pragma unroll
                for (int l = 0; l < 3; ++l) c[l] = cT[(t * 3 + l) * R + r];
                float4 *out = y_tri + (int64_t(r) * nt + t) * 3;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float gr = G[3 * k] * c[0].x + G[3 * k + 1] * c[1].x + G[3 * k + 2] * c[2].x;
                    const float gi = G[3 * k] * c[0].y + G[3 * k + 1] * c[1].y + G[3 * k + 2] * c[2].y;
                    out[k] = dd_zb(zr, zi, cl, gr, gi, DD{acc[k][j][v].x, 0.f}, DD{acc[k][j][v].y, 0.f});
                }
            }
    } else {
        double G[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) G[i] = __ldg(gram + 9 * t + i);
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int32_t r = rl + 32 * V * j + v;
                if (r >= R) continue;
                const double *cf = coef + int64_t(r) * (2 * ncond + 1);
                const double zr = cf[2 * cd], zi = cf[2 * cd + 1], cl = cf[2 * ncond];
                double2 c[3];
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    const C<T> u = cT[(t * 3 + l) * R + r];
                    c[l] = make_double2(double(u.x), double(u.y));
                }
                double2 *out = y_tri + (int64_t(r) * nt + t) * 3;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double gr = G[3 * k] * c[0].x + G[3 * k + 1] * c[1].x + G[3 * k + 2] * c[2].x;
                    const double gi = G[3 * k] * c[0].y + G[3 * k + 1] * c[1].y + G[3 * k + 2] * c[2].y;
                    const double fr = double(acc[k][j][v].x), fi = double(acc[k][j][v].y);
                    // Z_s * gram + j c_L * f
                    out[k] = make_double2(zr * gr - zi * gi - cl * fi, zr * gi + zi * gr + cl * fr);
                }
            }
    }
}

// Per triangle T and right-hand side r:
//   f_T[k] = sum_{T' near T} sum_l L_d(T,T')[k][l] c_T'[l]          (Eq. Lb, pre-corrected)
//          + sum_n sum_d W(n,T)[d][k] phi_g[d][n]                   (interpolation, I = B^T)
//   y_T[k] = Z_s sum_l G_T[k][l] c_T[l] + j c_L f_T[k]             (Eq. Zb, FP64)
// One warp per (T, slab of 32 V J right-hand sides), lanes over right-hand
// sides; each block record is read once per slab.  y_tri layout [R][nt][3].
template <typename T, int V, int J>
__global__ void __launch_bounds__(256)
    k_tri_gather(const int64_t *__restrict__ near_ptr, const Rec<T> *__restrict__ near_rec,
                 const int64_t *__restrict__ pt_ptr, const Rec<T> *__restrict__ pt_rec, const C<T> *__restrict__ cT,
                 const C<T> *__restrict__ phiT, const double *__restrict__ gram, const int32_t *__restrict__ cond,
                 const double *__restrict__ coef, const float2 *__restrict__ coef_dd, int ncond, int64_t nt,
                 int32_t R, int32_t nslab, TourE<T> *__restrict__ y_tri) {
    constexpr int SLAB = 32 * V * J;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= nt * nslab) return;
    const int64_t t = gw / nslab;
    const int32_t rbase = int32_t(gw % nslab) * SLAB;
    const int32_t rl = rbase + V * lane;
    C<T> acc[3][J][V];
    zero<T, V, J>(acc);
    if (rbase + SLAB <= R) {
        gather_rows<T, V, J, true>(near_rec, near_ptr[t], near_ptr[t + 1], cT, R, rl, acc);
        gather_rows<T, V, J, true>(pt_rec, pt_ptr[t], pt_ptr[t + 1], phiT, R, rl, acc);
    } else {
        gather_rows<T, V, J, false>(near_rec, near_ptr[t], near_ptr[t + 1], cT, R, rl, acc);
        gather_rows<T, V, J, false>(pt_rec, pt_ptr[t], pt_ptr[t + 1], phiT, R, rl, acc);
    }
    tri_epilogue<T, V, J>(acc, t, rl, R, cT, gram, cond, coef, coef_dd, ncond, nt, y_tri);
}

// The lossy kernel (pfft_params.kernel = SIE_KERNEL_LOSSY): as k_tri_gather with
// complex near blocks that depend on the frequency,
//   f_T[k] = sum_{T' near T} sum_l L_d,k(w_r)(T,T')[k][l] c_T'[l]
//          + sum_n sum_d W(n,T)[d][k] phi_g[d][n],
// Ltab[rslot[r]] being the blocks [n_near][3][3] of right-hand side r's
// frequency.  One warp per (T, slab of 32 J right-hand sides), one right-hand
// side per lane and load; lanes of one frequency read the same block.
template <typename T, int J>
__global__ void __launch_bounds__(256)
    k_tri_gather_lossy(const int64_t *__restrict__ near_ptr, const int32_t *__restrict__ near_col,
                       const C<T> *const *__restrict__ Ltab, const int32_t *__restrict__ rslot,
                       const int64_t *__restrict__ pt_ptr, const Rec<T> *__restrict__ pt_rec,
                       const C<T> *__restrict__ cT, const C<T> *__restrict__ phiT, const double *__restrict__ gram,
                       const int32_t *__restrict__ cond, const double *__restrict__ coef,
                       const float2 *__restrict__ coef_dd, int ncond, int64_t nt, int32_t R, int32_t nslab,
                       TourE<T> *__restrict__ y_tri) {
    constexpr int SLAB = 32 * J;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= nt * nslab) return;
    const int64_t t = gw / nslab;
    const int32_t rl = int32_t(gw % nslab) * SLAB + lane;
    C<T> acc[3][J][1];
    zero<T, 1, J>(acc);
    const C<T> *L[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int32_t r = rl + 32 * j;
        L[j] = r < R ? Ltab[rslot[r]] : nullptr;
    }
    const int64_t ld = 3 * int64_t(R);
    for (int64_t e = near_ptr[t]; e < near_ptr[t + 1]; ++e) {
        const C<T> *x = cT + int64_t(near_col[e]) * ld;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int32_t r = rl + 32 * j;
            if (r >= R) continue;
            const C<T> x0 = x[r], x1 = x[R + r], x2 = x[2 * R + r];
            const C<T> *b = L[j] + 9 * e;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const C<T> b0 = b[3 * k], b1 = b[3 * k + 1], b2 = b[3 * k + 2];
                acc[k][j][0].x += b0.x * x0.x - b0.y * x0.y + b1.x * x1.x - b1.y * x1.y + b2.x * x2.x - b2.y * x2.y;
                acc[k][j][0].y += b0.x * x0.y + b0.y * x0.x + b1.x * x1.y + b1.y * x1.x + b2.x * x2.y + b2.y * x2.x;
            }
        }
    }
    gather_rows<T, 1, J, false>(pt_rec, pt_ptr[t], pt_ptr[t + 1], phiT, R, rl, acc);
    tri_epilogue<T, 1, J>(acc, t, rl, R, cT, gram, cond, coef, coef_dd, ncond, nt, y_tri);
}

// Interpolated far field alone (mixed form, where the near blocks run on the
// tensor cores): ffar[T][k][r] = sum_n sum_d W(n,T)[d][k] phi_g[d][n].
template <typename T, int V, int J>
__global__ void __launch_bounds__(256)
    k_far_gather(const int64_t *__restrict__ pt_ptr, const Rec<T> *__restrict__ pt_rec,
                 const C<T> *__restrict__ phiT, int64_t nt, int32_t R, int32_t nslab, C<T> *__restrict__ ffar) {
    constexpr int SLAB = 32 * V * J;
    const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= nt * nslab) return;
    const int64_t t = gw / nslab;
    const int32_t rbase = int32_t(gw % nslab) * SLAB;
    const int32_t rl = rbase + V * lane;
    C<T> acc[3][J][V];
    zero<T, V, J>(acc);
    if (rbase + SLAB <= R) gather_rows<T, V, J, true>(pt_rec, pt_ptr[t], pt_ptr[t + 1], phiT, R, rl, acc);
    else gather_rows<T, V, J, false>(pt_rec, pt_ptr[t], pt_ptr[t + 1], phiT, R, rl, acc);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int32_t r = rl + 32 * V * j;
        if (r < R)
#pragma unroll
            for (int k = 0; k < 3; ++k) stv<T, V>(ffar + (t * 3 + k) * R + r, acc[k][j]);
    }
}

// y_b = sum over the branch's two triangles of s * y_T[k]; EO is the output
// element (complex128 for a branch-space result).
template <typename E, typename EO>
__global__ void k_branch_out(const E *__restrict__ y_tri, const int32_t *__restrict__ br_tri,
                             const int8_t *__restrict__ br_local, int64_t nt, int64_t nb, int64_t ldy, int32_t nrhs,
                             EO *__restrict__ y) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= ldy * nrhs) return;
    int64_t r = i / ldy, b = i % ldy;
    E v = ezero<E>();
    if (b < nb) {
        const E a = y_tri[(r * nt + br_tri[2 * b]) * 3 + br_local[2 * b]];
        const E c = y_tri[(r * nt + br_tri[2 * b + 1]) * 3 + br_local[2 * b + 1]];
        v = eadd(a, eneg(c));
    }
    EO o;
    eset(o, v);
    y[i] = o;
}

// Tour values for A: +delta(v) at v's enter slot, -delta(v) at its exit slot,
// delta(v) = voltage of v's parent twig walked from v towards the root.
// Grid (slots, right-hand-side groups of kTourRc), as k_tour_inject.
template <typename E>
__global__ void k_tour_voltage(const E *__restrict__ y_br, int64_t ldy, E *__restrict__ tour, int64_t nslots,
                               const int32_t *__restrict__ tour_node, const int8_t *__restrict__ tour_enter,
                               const int32_t *__restrict__ parent_branch, const int32_t *__restrict__ tail,
                               int32_t nrhs) {
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    const int32_t r0 = int32_t(blockIdx.y) * kTourRc;
    const int nr = min(kTourRc, nrhs - r0);
    const int v = tour_node[s];
    const int t = parent_branch[v];
    const bool neg = t >= 0 && ((tail[t] != v) != !tour_enter[s]);
    E d[kTourRc];
#pragma unroll
    for (int j = 0; j < kTourRc; ++j) {
        d[j] = ezero<E>();
        if (t >= 0 && j < nr) d[j] = y_br[int64_t(r0 + j) * ldy + t];
    }
#pragma unroll
    for (int j = 0; j < kTourRc; ++j)
        if (j < nr) tour[int64_t(r0 + j) * nslots + s] = neg ? eneg(d[j]) : d[j];
}

template <typename E>
__global__ void k_loop_out(const E *__restrict__ y_br, int64_t ldy, const E *__restrict__ P, int64_t nslots,
                           const int32_t *__restrict__ link_branch, const int32_t *__restrict__ tail,
                           const int32_t *__restrict__ head, const int32_t *__restrict__ enter, int64_t nl,
                           int32_t nrhs, double2 *__restrict__ y) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nl * nrhs) return;
    int64_t r = i / nl, l = i % nl;
    int32_t e = link_branch[l];
    const E *row = P + r * nslots;
    E v = y_br[r * ldy + e];
    v = eadd(v, row[enter[head[e]]]);
    v = eadd(v, eneg(row[enter[tail[e]]]));
    double2 o;
    eset(o, v);
    y[i] = o;
}

// Post-processing (Eq. CurT): current of every mesh branch, grid (branches, right-hand sides).
__global__ void k_branch_alpha(const double2 *__restrict__ x, int64_t nl, const double2 *__restrict__ P,
                               int64_t nslots, const int32_t *__restrict__ loop_of_branch,
                               const int32_t *__restrict__ twig_node, const int32_t *__restrict__ head,
                               const int32_t *__restrict__ enter, const int32_t *__restrict__ exit_, int64_t nb,
                               double2 *__restrict__ alpha) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int64_t r = blockIdx.y;
    alpha[r * nb + b] = branch_current<double>(int32_t(b), r, x, nl, P, nslots, loop_of_branch, twig_node, head,
                                               enter, exit_);
}

// Post-processing: panel potential = root-path sum of the panel's node minus that
// of its conductor's reference node, grid (panels, right-hand sides).
__global__ void k_panel_phi(const double2 *__restrict__ P, int64_t nslots, const int32_t *__restrict__ slot,
                            const int32_t *__restrict__ ref, int64_t nt, double2 *__restrict__ phi) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int64_t r = blockIdx.y;
    const double2 *row = P + r * nslots;
    phi[r * nt + t] = csub(row[slot[t]], row[ref[t]]);
}

inline unsigned nblk(int64_t n, int t = 256) { return unsigned((n + t - 1) / t); }

}  // namespace

namespace sie {

// Grows the matvec scratch to hold nrhs right-hand sides in precision `prec`.
// Buffers only grow: a plan used in both precisions keeps FP64-sized buffers
// (the mixed form reads them as complex64) and the mixed form's far-field
// buffer, so alternating precisions (iterative refinement) never reallocates.
int scratch_reserve(pfft_plan *p, int32_t nrhs, int prec) {
    Scratch &s = p->scr;
    // complex values of the field steps: complex64 in the mixed form, 16 bytes
    // (complex128 or complex double-float) otherwise
    const bool mixed = prec == SIE_PREC_MIXED;
    const int want_cs = mixed ? int(sizeof(float2)) : int(sizeof(double2));
    if (s.cap_rhs >= nrhs && s.cs >= want_cs && (!mixed || s.ffar)) return SIE_OK;
    const int64_t R = std::max<int64_t>({int64_t(nrhs), int64_t(s.cap_rhs), 1});
    const size_t cs = size_t(std::max(want_cs, s.cs));
    const bool with_far = mixed || s.ffar != nullptr;
    for (void *a : {s.tour, s.grid, s.spec, s.phiT, s.y_tri, s.y_br, (void *)s.coef, s.cT, s.ffar})
        if (a) cudaFree(a);
    s = Scratch{};
    constexpr int kBufs = 9;
    const size_t sizes[kBufs] = {
        size_t(R) * 2 * p->nn * sizeof(double2),
        size_t(R) * 3 * p->Ng * cs,
        size_t(R) * 3 * p->Mx * (p->Ny + (p->large_plane ? p->My : 0)) * p->Nz * cs,
        size_t(R) * 3 * p->Ng * cs,
        size_t(R) * p->nt * 3 * sizeof(double2),
        size_t(R) * (p->nb + p->np) * sizeof(double2),
        size_t(R) * (2 * p->ncond + 1) * (sizeof(double) + sizeof(float2)),
        size_t(R) * p->nt * 3 * cs,
        with_far ? size_t(R) * p->nt * 3 * sizeof(float2) : 0};
    void **dst[kBufs] = {&s.tour, &s.grid, &s.spec, &s.phiT, &s.y_tri, &s.y_br, (void **)&s.coef, &s.cT,
                         &s.ffar};
    for (int i = 0; i < kBufs; ++i) {
        if (!sizes[i]) continue;
        cudaError_t e = cudaMalloc(dst[i], sizes[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) if (*dst[j]) { cudaFree(*dst[j]); *dst[j] = nullptr; }
            set_error(std::string("scratch allocation failed: ") + cudaGetErrorString(e));
            s = Scratch{};
            return SIE_ERR_OOM;
        }
        s.bytes += sizes[i];
    }
    s.cap_rhs = int32_t(R);
    s.cs = int(cs);
    ++p->scr_gen;
    return SIE_OK;
}

// Block-sparse stages for one slab shape: V complex per load, J loads per lane.
template <typename T, int V, int J> struct Blocks {
    static constexpr int SLAB = 32 * V * J;
    static const Rec<T> *pn(const pfft_plan *p) {
        if constexpr (is_df<T>) return p->d_pn_recdf;
        else if constexpr (is_f64<T>) return p->d_pn_rec64;
        else return p->d_pn_rec32;
    }
    static const Rec<T> *pt(const pfft_plan *p) {
        if constexpr (is_df<T>) return p->d_pt_recdf;
        else if constexpr (is_f64<T>) return p->d_pt_rec64;
        else return p->d_pt_rec32;
    }
    static const Rec<T> *nr(const pfft_plan *p) {
        if constexpr (is_df<T>) return p->d_near_recdf;
        else if constexpr (is_f64<T>) return p->d_near_rec64;
        else return p->d_near_rec32;
    }
    static int project(pfft_plan *p, int32_t R, cudaStream_t st) {
        const dim3 grid(unsigned((p->Ng + kProjNodes - 1) / kProjNodes), unsigned((R + SLAB - 1) / SLAB));
        k_project<T, V, J><<<grid, 32 * kProjNodes, proj_smem<T, V, J>(), st>>>(
            p->d_pn_ptr, pn(p), (const C<T> *)p->scr.cT, p->Ng, R, (C<T> *)p->scr.grid);
        SIE_LAUNCH_CHECK(p);
        return SIE_OK;
    }
    static int far_gather(pfft_plan *p, int32_t R, cudaStream_t st) {
        const int32_t nslab = (R + SLAB - 1) / SLAB;
        const int64_t warps = p->nt * nslab;
        k_far_gather<T, V, J><<<unsigned((warps * 32 + 255) / 256), 256, 0, st>>>(
            p->d_pt_ptr, pt(p), (const C<T> *)p->scr.phiT, p->nt, R, nslab, (C<T> *)p->scr.ffar);
        SIE_LAUNCH_CHECK(p);
        return SIE_OK;
    }
    static int tri_gather_lossy(pfft_plan *p, int32_t R, cudaStream_t st) {
        static_assert(V == 1 && !is_df<T>, "one right-hand side per lane and load; FP64 or mixed");
        const int32_t nslab = (R + SLAB - 1) / SLAB;
        const int64_t warps = p->nt * nslab;
        const int prec = is_f64<T> ? SIE_PREC_FP64 : SIE_PREC_MIXED;
        k_tri_gather_lossy<T, J><<<unsigned((warps * 32 + 255) / 256), 256, 0, st>>>(
            p->d_near_ptr, p->d_near_col, reinterpret_cast<const C<T> *const *>(lossy_ltab(p, prec)),
            lossy_rslot(p), p->d_pt_ptr, pt(p), (const C<T> *)p->scr.cT, (const C<T> *)p->scr.phiT, p->d_gram,
            p->d_cond, p->scr.coef, coef_dd(p), p->ncond, p->nt, R, nslab, (TourE<T> *)p->scr.y_tri);
        SIE_LAUNCH_CHECK(p);
        return SIE_OK;
    }
    static int tri_gather(pfft_plan *p, int32_t R, cudaStream_t st) {
        const int32_t nslab = (R + SLAB - 1) / SLAB;
        const int64_t warps = p->nt * nslab;
        k_tri_gather<T, V, J><<<unsigned((warps * 32 + 255) / 256), 256, 0, st>>>(
            p->d_near_ptr, nr(p), p->d_pt_ptr, pt(p), (const C<T> *)p->scr.cT, (const C<T> *)p->scr.phiT,
            p->d_gram, p->d_cond, p->scr.coef, coef_dd(p), p->ncond, p->nt, R, nslab, (TourE<T> *)p->scr.y_tri);
        SIE_LAUNCH_CHECK(p);
        return SIE_OK;
    }
};

// Slab shape per right-hand-side count: a warp serves one triangle (or node)
// and 32 V J right-hand sides, V complex per load (FP32: two per 16-byte load
// when R is even, so that rows of [.][3][R] start on 16-byte boundaries), J
// loads per lane; the smallest slab that covers R keeps every lane busy.
#define SIE_SLAB_DISPATCH(T, R, CALL)                                                     \
    do {                                                                                 \
        if constexpr (is_df<T>) {                                                         \
            if ((R) <= 32) return Blocks<df, 1, 1>::CALL;                                 \
            return Blocks<df, 1, 2>::CALL;                                                \
        } else if constexpr (is_f64<T>) {                                                 \
            if ((R) <= 32) return Blocks<double, 1, 1>::CALL;                             \
            return Blocks<double, 1, 2>::CALL;                                            \
        } else {                                                                          \
            if ((R) <= 32) return Blocks<float, 1, 1>::CALL;                              \
            if ((R) <= 64) return (R) % 2 == 0 ? Blocks<float, 2, 1>::CALL : Blocks<float, 1, 2>::CALL; \
            return (R) % 2 == 0 ? Blocks<float, 2, 2>::CALL : Blocks<float, 1, 4>::CALL;  \
        }                                                                                 \
    } while (0)
// The far-field gather keeps slabs at most 64 wide in FP32: its 128-wide form
// needs 80 registers a thread, which caps residency at 3 CTAs per SM for this
// latency-bound gather; two 64-wide slabs (61 registers) read each block record
// twice but keep 4 CTAs resident (measured: 0.77 -> 0.66 ms on the bond-wire
// step; the projection, whose block records dominate its loads, is faster 128
// wide).
#define SIE_SLAB_DISPATCH_NARROW(T, R, CALL)                                              \
    do {                                                                                 \
        if constexpr (is_f32<T>) {                                                        \
            if ((R) > 32) return (R) % 2 == 0 ? Blocks<float, 2, 1>::CALL : Blocks<float, 1, 2>::CALL; \
        }                                                                                 \
        SIE_SLAB_DISPATCH(T, R, CALL);                                                    \
    } while (0)
template <typename T> int run_project(pfft_plan *p, int32_t R, cudaStream_t st) {
    if constexpr (is_f32<T>) {
        // mixed form: staged node chunks when asked for (pfft_plan_set_kernel_tuning,
        // the autotuner); the direct gather is the default (measured on the bond
        // wires at 128 right-hand sides: 0.68 ms direct against 1.28 ms staged, whose
        // 32-wide slabs read each block record four times as often)
        if (p->n_pchunk > 0 && p->kt.proj_slab == kChunkRhs) {
            if (p->n_pchunk > INT32_MAX) return fail(SIE_ERR_ARG, "projection: too many node chunks");
            if (int rc = set_smem((const void *)k_project_tiled, kPTSmem)) return rc;
            const dim3 grid(unsigned(p->n_pchunk), unsigned((R + kChunkRhs - 1) / kChunkRhs));
            k_project_tiled<<<grid, 256, kPTSmem, st>>>(p->d_pch_node_ptr, p->d_pch_nodes, p->d_pch_tri_ptr,
                                                        p->d_pch_tri, p->d_pn_ptr, p->d_pn_rec32, p->d_pn_lcol,
                                                        (const float2 *)p->scr.cT, p->Ng, R, (float2 *)p->scr.grid);
            SIE_LAUNCH_CHECK(p);
            return SIE_OK;
        }
    }
    if (p->kt.proj_slab == 64) SIE_SLAB_DISPATCH_NARROW(T, R, project(p, R, st));
    SIE_SLAB_DISPATCH(T, R, project(p, R, st));
}
int run_far_gather(pfft_plan *p, int32_t R, cudaStream_t st) {
    if (p->kt.far_slab == 128) SIE_SLAB_DISPATCH(float, R, far_gather(p, R, st));
    SIE_SLAB_DISPATCH_NARROW(float, R, far_gather(p, R, st));
}
template <typename T> int run_tri_gather(pfft_plan *p, int32_t R, cudaStream_t st) {
    SIE_SLAB_DISPATCH(T, R, tri_gather(p, R, st));
}
template <typename T> int run_tri_gather_lossy(pfft_plan *p, int32_t R, cudaStream_t st) {
    if (R <= 32) return Blocks<T, 1, 1>::tri_gather_lossy(p, R, st);
    if (R <= 64) return Blocks<T, 1, 2>::tri_gather_lossy(p, R, st);
    return Blocks<T, 1, 4>::tri_gather_lossy(p, R, st);
}

// Smallest right-hand-side count for the tensor-core near field (mixed form).
constexpr int32_t kNearMmaMinRhs = 96;

template <typename T>
int matvec_t(pfft_plan *p, const double2 *x, double2 *y, int32_t R, int space, cudaStream_t st) {
    Scratch &s = p->scr;
    const int64_t nslots = 2 * p->nn;
    const int64_t ldy = p->nb + p->np;
    using E = TourE<T>;
    E *tour = (E *)s.tour;
    E *y_tri = (E *)s.y_tri, *y_br = (E *)s.y_br;
    std::unique_ptr<StageTimer> tm(new StageTimer(p, SIE_STAGE_LOOP_TO_BRANCH, st));
    if (space == SIE_SPACE_LOOP) {
        k_tour_inject<<<dim3(nblk(nslots), unsigned((R + kTourRc - 1) / kTourRc)), 256, 0, st>>>(
            x, p->nl, tour, nslots, p->d_tour_node, p->d_tour_enter, p->d_nl_ptr, p->d_nl_loop, p->d_nl_sign, R);
        SIE_LAUNCH_CHECK(p);
        k_scan_rows<E><<<R, 1024, 0, st>>>(tour, nslots);
        SIE_LAUNCH_CHECK(p);
    }
    k_alpha_tri<T><<<nblk(p->nt * R), 256, 0, st>>>(x, p->nl, tour, nslots, p->d_tb, p->d_ts, p->d_loop_of_branch,
                                                     p->d_twig_node, p->d_head, p->d_enter, p->d_exit, p->nt, R, space,
                                                     p->nb, (C<T> *)s.cT);
    SIE_LAUNCH_CHECK(p);
    tm.reset(new StageTimer(p, SIE_STAGE_PROJECT, st));
    int rc = run_project<T>(p, R, st);
    if (rc) return rc;
    tm.reset();
    const int prec = is_df<T> ? SIE_PREC_DF : is_f64<T> ? SIE_PREC_FP64 : SIE_PREC_MIXED;
    const bool lossy = !is_df<T> && p->params.kernel == SIE_KERNEL_LOSSY;
    rc = fft_conv(p, s.grid, s.spec, R, prec, st, lossy ? lossy_sel(p, prec) : nullptr);
    if (rc) return rc;
    tm.reset(new StageTimer(p, SIE_STAGE_INTERP, st));
    {
        const int32_t B = 3 * R;
        const dim3 grid(unsigned(p->n_tiles), unsigned((B + 31) / 32));
        k_regroup<T><<<grid, 256, 0, st>>>((const C<T> *)s.grid, p->d_tiles, p->Ng, B, (C<T> *)s.phiT);
        SIE_LAUNCH_CHECK(p);
    }
    // mixed form, R even and at least kNearMmaMinRhs: near blocks on the tensor
    // cores (their operand rows are 16-byte aligned only for even R; a 128-column
    // slab costs the same however few of its columns are used, so below about
    // three quarters of a slab the CUDA-core gather is faster); otherwise one
    // CUDA-core gather
    if constexpr (is_df<T>) {
        tm.reset(new StageTimer(p, SIE_STAGE_NEAR, st));
        rc = run_tri_gather<T>(p, R, st);       // near + interpolation + y_T in one gather
    } else if (lossy) {
        // complex near blocks per frequency: one CUDA-core gather (near + interpolation + y_T)
        tm.reset(new StageTimer(p, SIE_STAGE_NEAR, st));
        rc = run_tri_gather_lossy<T>(p, R, st);
    } else if (is_f32<T> && R % 2 == 0 && p->kt.near != 2 && (R >= kNearMmaMinRhs || p->kt.near == 1)) {
        rc = run_far_gather(p, R, st);          // interpolation (step 3) on the CUDA cores
        if (rc) return rc;
        tm.reset(new StageTimer(p, SIE_STAGE_NEAR, st));
        rc = near_mma_launch(p, R, st);         // near blocks on the tensor cores + y_T
    } else {
        tm.reset(new StageTimer(p, SIE_STAGE_NEAR, st));
        rc = run_tri_gather<T>(p, R, st);       // near + interpolation + y_T in one gather
    }
    if (rc) return rc;
    tm.reset(new StageTimer(p, SIE_STAGE_BRANCH_TO_LOOP, st));
    if (space == SIE_SPACE_BRANCH) {
        k_branch_out<E, double2><<<nblk(p->nb * R), 256, 0, st>>>(y_tri, p->d_br_tri, p->d_br_local, p->nt, p->nb,
                                                                  p->nb, R, y);
        SIE_LAUNCH_CHECK(p);
        return SIE_OK;
    }
    k_branch_out<E, E><<<nblk(ldy * R), 256, 0, st>>>(y_tri, p->d_br_tri, p->d_br_local, p->nt, p->nb, ldy, R,
                                                        y_br);
    SIE_LAUNCH_CHECK(p);
    k_tour_voltage<E><<<dim3(nblk(nslots), unsigned((R + kTourRc - 1) / kTourRc)), 256, 0, st>>>(
        y_br, ldy, tour, nslots, p->d_tour_node, p->d_tour_enter, p->d_parent_branch, p->d_tail, R);
    SIE_LAUNCH_CHECK(p);
    k_scan_rows<E><<<R, 1024, 0, st>>>(tour, nslots);
    SIE_LAUNCH_CHECK(p);
    k_loop_out<E><<<nblk(p->nl * R), 256, 0, st>>>(y_br, ldy, tour, nslots, p->d_link_branch, p->d_tail, p->d_head,
                                                    p->d_enter, p->nl, R, y);
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

float2 *coef_dd(const pfft_plan *p) {
    return reinterpret_cast<float2 *>(p->scr.coef + size_t(p->scr.cap_rhs) * (2 * p->ncond + 1));
}

std::complex<double> surface_impedance(const pfft_plan *p, int c, double w) {
    using cd = std::complex<double>;
    const double sig = p->sigma[c], t = p->t_eff.empty() ? 0.0 : p->t_eff[c];
    if (!(t > 0.0)) return cd(1.0, 1.0) * std::sqrt(w * kMu0 / (2.0 * sig));
    const cd gamma = cd(1.0, 1.0) * std::sqrt(w * kMu0 * sig / 2.0);
    const cd z = gamma * (t / 2.0);
    // z coth z: Taylor series for small |z|, else coth from exp(-2z) (Re z >= 0)
    cd zc;
    if (std::abs(z) < 1e-2) {
        const cd z2 = z * z;
        zc = 1.0 + z2 / 3.0 - z2 * z2 / 45.0;
    } else {
        const cd e = std::exp(-2.0 * z);
        zc = z * (1.0 + e) / (1.0 - e);
    }
    return 2.0 / (sig * t) * zc;
}

// Per right-hand side: Z_s of each conductor and c_L / j (Eq. ImpedanceOp, Eq. Zb),
// in FP64 and as double-float pairs.
int fill_coef(const pfft_plan *p, const double *omega, int32_t R, double *cf, float2 *cd) {
    const size_t n = size_t(R) * (2 * p->ncond + 1);
    for (int32_t r = 0; r < R; ++r) {
        const double w = omega[r];
        if (!(w >= 0.0) || !std::isfinite(w)) return fail(SIE_ERR_ARG, "pfft_matvec: omega must be finite and >= 0");
        for (int c = 0; c < p->ncond; ++c) {
            const std::complex<double> zs = surface_impedance(p, c, w);
            cf[r * (2 * p->ncond + 1) + 2 * c] = zs.real();
            cf[r * (2 * p->ncond + 1) + 2 * c + 1] = zs.imag();
        }
        cf[r * (2 * p->ncond + 1) + 2 * p->ncond] = w * kMu0 / (4.0 * M_PI);
    }
    for (size_t i = 0; i < n; ++i) {
        const float hi = float(cf[i]);
        cd[i] = make_float2(hi, float(cf[i] - double(hi)));
    }
    return SIE_OK;
}

int upload_coef(pfft_plan *p, const double *omega, int32_t R, cudaStream_t st) {
    const size_t n = size_t(R) * (2 * p->ncond + 1);
    std::vector<double> cf(n);
    std::vector<float2> cd(n);
    int rc = fill_coef(p, omega, R, cf.data(), cd.data());
    if (rc) return rc;
    SIE_CUDA(cudaMemcpyAsync(p->scr.coef, cf.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    SIE_CUDA(cudaMemcpyAsync(coef_dd(p), cd.data(), n * sizeof(float2), cudaMemcpyHostToDevice, st));
    return SIE_OK;
}

int matvec_async(pfft_plan *p, const void *x, void *y, int32_t nrhs, const double *omega, int space, int prec,
                 cudaStream_t st) {
    int rc = scratch_reserve(p, nrhs, prec);
    if (rc) return rc;
    rc = upload_coef(p, omega, nrhs, st);
    if (rc) return rc;
    if (p->params.kernel == SIE_KERNEL_LOSSY && (rc = lossy_prepare(p, omega, nrhs, st))) return rc;
    if (prec == SIE_PREC_DF && (rc = df_prepare(p, st))) return rc;
    return matvec_launch(p, x, y, nrhs, space, prec, st);
}

int matvec_launch(pfft_plan *p, const void *x, void *y, int32_t nrhs, int space, int prec, cudaStream_t st) {
    if (prec == SIE_PREC_FP64)
        return matvec_t<double>(p, (const double2 *)x, (double2 *)y, nrhs, space, st);
    if (prec == SIE_PREC_DF) {
        if (!p->df_ready || p->params.kernel != SIE_KERNEL_STATIC)
            return fail(SIE_ERR_ARG, "double-float product: static kernel plans only, tables built first");
        return matvec_t<df>(p, (const double2 *)x, (double2 *)y, nrhs, space, st);
    }
    return matvec_t<float>(p, (const double2 *)x, (double2 *)y, nrhs, space, st);
}

}  // namespace sie

extern "C" int pfft_matvec(pfft_plan *p, const void *x, void *y, int32_t nrhs, const double *omega, int32_t space,
                           int32_t prec, void *cuda_stream) {
    if (!p || !x || !y || !omega) return fail(SIE_ERR_ARG, "pfft_matvec: NULL argument");
    if (nrhs < 1) return fail(SIE_ERR_ARG, "pfft_matvec: nrhs must be >= 1");
    if (space != SIE_SPACE_LOOP && space != SIE_SPACE_BRANCH) return fail(SIE_ERR_ARG, "pfft_matvec: bad space");
    if (prec != SIE_PREC_FP64 && prec != SIE_PREC_MIXED && prec != SIE_PREC_DF)
        return fail(SIE_ERR_ARG, "pfft_matvec: bad precision");
    if (prec == SIE_PREC_DF && p->params.kernel != SIE_KERNEL_STATIC)
        return fail(SIE_ERR_ARG, "pfft_matvec: the double-float product takes the static kernel only");
    const int64_t n = space == SIE_SPACE_LOOP ? p->nl : p->nb;
    const char *xb = (const char *)x, *yb = (const char *)y;
    const size_t bytes = size_t(nrhs) * n * sizeof(double2);
    if (xb < yb + bytes && yb < xb + bytes) return fail(SIE_ERR_ARG, "pfft_matvec: x and y overlap");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    (void)cudaGetLastError();   // clear a stale error left by earlier work in this thread
    int rc = sie::matvec_async(p, x, y, nrhs, omega, space, prec, st);
    if (rc) return rc;
    return sie::finish_call(p, st);
}

extern "C" int sie_postprocess(pfft_plan *p, const void *x, int32_t nrhs, const double *omega, int32_t prec,
                               void *i_branch, void *v_branch, void *phi, void *cuda_stream) {
    using namespace sie;
    if (!p || !x || nrhs < 1) return fail(SIE_ERR_ARG, "sie_postprocess: bad argument");
    if (prec != SIE_PREC_FP64 && prec != SIE_PREC_MIXED) return fail(SIE_ERR_ARG, "sie_postprocess: bad precision");
    if ((v_branch || phi) && !omega) return fail(SIE_ERR_ARG, "sie_postprocess: omega is needed for voltages");
    if (!i_branch && !v_branch && !phi) return SIE_OK;
    if (nrhs > 65535) return fail(SIE_ERR_ARG, "sie_postprocess: at most 65535 right-hand sides per call");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    (void)cudaGetLastError();
    const int64_t nb = p->nb, nt = p->nt, nslots = 2 * p->nn, R = nrhs;
    int rc = scratch_reserve(p, nrhs, prec);   // the size the product below uses: no later regrowth
    if (rc) return rc;
    // temporaries for outputs the caller did not ask for but later steps need
    double2 *alpha = static_cast<double2 *>(i_branch), *vb = static_cast<double2 *>(v_branch);
    double2 *tmp_a = nullptr, *tmp_v = nullptr;
    auto cleanup = [&]() {
        if (tmp_a) cudaFree(tmp_a);
        if (tmp_v) cudaFree(tmp_v);
    };
    if (!alpha) {
        if (cudaMalloc((void **)&tmp_a, size_t(R) * nb * sizeof(double2)) != cudaSuccess)
            return fail(SIE_ERR_OOM, "sie_postprocess: out of device memory");
        alpha = tmp_a;
    }
    if (phi && !vb) {
        if (cudaMalloc((void **)&tmp_v, size_t(R) * nb * sizeof(double2)) != cudaSuccess) {
            cleanup();
            return fail(SIE_ERR_OOM, "sie_postprocess: out of device memory");
        }
        vb = tmp_v;
    }
    double2 *tour = static_cast<double2 *>(p->scr.tour);
    const dim3 gs(nblk(nslots), unsigned((R + kTourRc - 1) / kTourRc)), gb(nblk(nb), unsigned(R)),
        gt(nblk(nt), unsigned(R));
    // branch currents: alpha = A^T x through the tour prefix sums (FP64)
    k_tour_inject<double2><<<gs, 256, 0, st>>>(static_cast<const double2 *>(x), p->nl, tour, nslots, p->d_tour_node,
                                               p->d_tour_enter, p->d_nl_ptr, p->d_nl_loop, p->d_nl_sign, R);
    k_scan_rows<double2><<<unsigned(R), 1024, 0, st>>>(tour, nslots);
    k_branch_alpha<<<gb, 256, 0, st>>>(static_cast<const double2 *>(x), p->nl, tour, nslots, p->d_loop_of_branch,
                                       p->d_twig_node, p->d_head, p->d_enter, p->d_exit, nb, alpha);
    p->launches += 3;
    if (cudaGetLastError() != cudaSuccess) { cleanup(); return fail(SIE_ERR_CUDA, "sie_postprocess: launch failed"); }
    if (vb) {   // branch voltage drops: the branch-space product Z_b alpha
        rc = matvec_async(p, alpha, vb, nrhs, omega, SIE_SPACE_BRANCH, prec, st);
        if (rc) { cleanup(); return rc; }
    }
    if (phi) {   // potentials: root-path sums of the twig drops, minus the reference node's
        k_tour_voltage<double2><<<gs, 256, 0, st>>>(vb, nb, tour, nslots, p->d_tour_node, p->d_tour_enter,
                                                     p->d_parent_branch, p->d_tail, R);
        k_scan_rows<double2><<<unsigned(R), 1024, 0, st>>>(tour, nslots);
        k_panel_phi<<<gt, 256, 0, st>>>(tour, nslots, p->d_panel_slot, p->d_panel_ref, nt,
                                        static_cast<double2 *>(phi));
        p->launches += 3;
        if (cudaGetLastError() != cudaSuccess) { cleanup(); return fail(SIE_ERR_CUDA, "sie_postprocess: launch failed"); }
    }
    const cudaError_t e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return fail(SIE_ERR_CUDA, std::string("sie_postprocess: ") + cudaGetErrorString(e));
    return check_device_errors(p);
}
