// Sparse direct factorisation of the preconditioner's nodal Laplacian by
// nested dissection (multifrontal LDL^T), for conductors whose reverse
// Cuthill-McKee band is too wide for the band factorisation (plates and
// planes: thousands of unknowns across).
//
// Eq. (Precond) asks for a direct factorisation of P = A diag(Z_b) A^T (the
// paper uses a sparse direct solver).  P^-1 is applied through the nodal form
// of the same circuit (sie_solve.cu): K u = rhs with K the Laplacian of the
// branch admittances 1/D_e, complex symmetric, its Hermitian part positive
// definite, so LDL^T without pivoting exists.  Here K is ordered by nested
// dissection and factorised front by front:
//
//   ordering (host, once per plan): the unknowns are split at the median of
//     their centroids along the longest axis of their box; the nodes of the
//     smaller side of the cut that touch the other side form the separator,
//     numbered after both halves, which are split again down to leaves of at
//     most kLeaf unknowns.  The elimination tree is the tree of separators;
//     front f holds its pivots I_f (contiguous indices) and the later
//     unknowns U_f its subtree couples to (sorted).
//   numeric (device, per frequency): the fronts of one tree level at a time,
//     deepest first: assemble F_f = [K(I_f, I_f ∪ U_f)] + the update matrices
//     of its children (extend-add), then F_f = L D L^T on its pivots in panels
//     of 32 columns (one CTA factors a panel, a tiled update applies it to the
//     trailing lower triangle), leaving the Schur complement on U_f for the
//     parent.  Fronts are dense, column-major, lower triangle only.
//   solve (device): forward through the levels (each front gathers its
//     children's update vectors, eliminates its pivots, passes its update
//     vector up), then backward from the root (each front gathers the final
//     values of U_f, then solves with L^T), with 1/d in between.
//
// Everything is deterministic: no atomics, children added in a fixed order.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "sie_plan.h"

namespace sie {

namespace {
constexpr int kLeaf = 128;      // largest leaf of the dissection
constexpr int kPanel = 32;      // columns per factorisation panel
constexpr int kTile = 32;       // trailing-update tile
}  // namespace

struct NdState {
    int32_t nfront = 0;
    int64_t nunk = 0;
    int64_t sumF = 0, sumL = 0, sumU = 0;   // front workspace, factor and update-vector sizes
    int32_t max_nf = 0;
    int64_t flops = 0;                      // complex multiply-adds of one factorisation
    std::vector<int32_t> level_ptr;         // fronts of level h: order[level_ptr[h] .. level_ptr[h+1])
    std::vector<int32_t> level_max_nv, level_max_nf;
    // device
    int32_t *order = nullptr;               // fronts grouped by level
    int64_t *first = nullptr, *Foff = nullptr, *Loff = nullptr, *Uoff = nullptr;
    int32_t *nv = nullptr, *nf = nullptr;
    int32_t *child_ptr = nullptr, *child = nullptr;
    int32_t *uidx = nullptr, *relpos = nullptr;   // [sumU]: U_f (global) and their positions in the parent
    int32_t *row_loc = nullptr;             // per row entry of the Laplacian: position in its front (-1: none)
    std::vector<void *> allocs;
};

namespace {

template <typename T>
int nd_upload(NdState *s, T **dst, const std::vector<T> &v) {
    const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    SIE_CUDA(cudaMalloc((void **)dst, bytes));
    s->allocs.push_back(*dst);
    if (!v.empty()) SIE_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SIE_OK;
}

struct Node {
    int64_t first = 0;
    int32_t nv = 0;
    std::vector<int32_t> children;
};

struct Dissect {
    const std::vector<std::vector<int32_t>> &adj;
    const std::vector<double> &xyz;
    std::vector<int32_t> &perm;
    std::vector<Node> &tree;
    std::vector<int8_t> side;

    // Orders S (raw unknown ids); returns its tree node, -1 when S is empty.
    int rec(std::vector<int32_t> S) {
        if (S.empty()) return -1;
        if (S.size() <= size_t(kLeaf)) return leaf(S);
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int32_t v : S)
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], xyz[3 * size_t(v) + d]);
                hi[d] = std::max(hi[d], xyz[3 * size_t(v) + d]);
            }
        int ax = 0;
        for (int d = 1; d < 3; ++d)
            if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
        const size_t h = S.size() / 2;
        std::nth_element(S.begin(), S.begin() + h, S.end(), [&](int32_t a, int32_t b) {
            const double xa = xyz[3 * size_t(a) + ax], xb = xyz[3 * size_t(b) + ax];
            return xa != xb ? xa < xb : a < b;
        });
        for (size_t k = 0; k < S.size(); ++k) side[S[k]] = k < h ? 1 : 2;
        std::vector<int32_t> sepA, sepB;
        for (size_t k = 0; k < S.size(); ++k) {
            const int32_t v = S[k];
            const int8_t other = side[v] == 1 ? 2 : 1;
            for (int32_t w : adj[v])
                if (side[w] == other) {
                    (side[v] == 1 ? sepA : sepB).push_back(v);
                    break;
                }
        }
        const bool takeA = sepA.size() <= sepB.size();
        std::vector<int32_t> &sep = takeA ? sepA : sepB;
        for (int32_t v : sep) side[v] = 3;
        std::vector<int32_t> A, B;
        for (int32_t v : S) {
            if (side[v] == 1) A.push_back(v);
            else if (side[v] == 2) B.push_back(v);
        }
        for (int32_t v : S) side[v] = 0;
        std::sort(sep.begin(), sep.end());
        std::vector<int32_t>().swap(S);
        const int ca = rec(std::move(A));
        const int cb = rec(std::move(B));
        Node n;
        n.first = int64_t(perm.size());
        n.nv = int32_t(sep.size());
        if (ca >= 0) n.children.push_back(ca);
        if (cb >= 0) n.children.push_back(cb);
        perm.insert(perm.end(), sep.begin(), sep.end());
        tree.push_back(std::move(n));
        return int(tree.size()) - 1;
    }

    int leaf(std::vector<int32_t> &S) {
        std::sort(S.begin(), S.end());
        Node n;
        n.first = int64_t(perm.size());
        n.nv = int32_t(S.size());
        perm.insert(perm.end(), S.begin(), S.end());
        tree.push_back(std::move(n));
        return int(tree.size()) - 1;
    }
};

// ---------------------------------------------------------------- numeric kernels

struct FrontArgs {
    const int32_t *order;
    const int64_t *first, *Foff, *Loff, *Uoff;
    const int32_t *nv, *nf;
    const int32_t *child_ptr, *child, *uidx, *relpos;
};

// F_f = K(I_f, I_f ∪ U_f) (lower triangle, column-major, leading dimension nf)
// plus the children's update matrices F_c[nv_c:, nv_c:].
__global__ void k_nd_assemble(FrontArgs fa, int32_t lvl0, const double2 *__restrict__ a,
                              const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ row_br,
                              const int32_t *__restrict__ row_loc, double2 *__restrict__ W) {
    const int32_t f = fa.order[lvl0 + blockIdx.x];
    const int32_t nf = fa.nf[f], nv = fa.nv[f];
    double2 *F = W + fa.Foff[f];
    for (int64_t t = threadIdx.x; t < int64_t(nf) * nf; t += blockDim.x) F[t] = make_double2(0.0, 0.0);
    __syncthreads();
    // the original entries: each thread owns the columns of its pivots
    for (int32_t li = threadIdx.x; li < nv; li += blockDim.x) {
        const int64_t i = fa.first[f] + li;
        double2 d = make_double2(0.0, 0.0);
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const double2 w = a[row_br[k]];
            d = cadd(d, w);
            const int32_t loc = row_loc[k];
            if (loc >= 0) F[int64_t(li) * nf + loc] = csub(F[int64_t(li) * nf + loc], w);
        }
        F[int64_t(li) * nf + li] = cadd(F[int64_t(li) * nf + li], d);
    }
    // extend-add, one child at a time
    for (int32_t q = fa.child_ptr[f]; q < fa.child_ptr[f + 1]; ++q) {
        __syncthreads();
        const int32_t c = fa.child[q];
        const int32_t nfc = fa.nf[c], nvc = fa.nv[c], mc = nfc - nvc;
        const double2 *U = W + fa.Foff[c] + int64_t(nvc) * nfc + nvc;
        const int32_t *rp = fa.relpos + fa.Uoff[c];
        for (int64_t t = threadIdx.x; t < int64_t(mc) * mc; t += blockDim.x) {
            const int32_t r = int32_t(t % mc), cc = int32_t(t / mc);
            if (r < cc) continue;
            double2 &dst = F[int64_t(rp[cc]) * nf + rp[r]];
            dst = cadd(dst, U[int64_t(cc) * nfc + r]);
        }
    }
}

// Panel [p, p + 32) of each front of the level: for each pivot column c the
// multipliers l_ic = F_ic / d_c (i > c), and the panel's later columns
// F_ic' -= l_ic F_c'c (i >= c' > c).  The diagonal keeps d_c.
__global__ void k_nd_panel(FrontArgs fa, int32_t lvl0, int32_t p, double2 *__restrict__ W, int *status) {
    const int32_t f = fa.order[lvl0 + blockIdx.x];
    const int32_t nf = fa.nf[f], nv = fa.nv[f];
    if (nv <= p) return;
    const int32_t pe = min(p + kPanel, nv);
    double2 *F = W + fa.Foff[f];
    __shared__ double2 wc[kPanel];
    for (int32_t c = p; c < pe; ++c) {
        __syncthreads();
        const double2 d = F[int64_t(c) * nf + c];
        if (d.x == 0.0 && d.y == 0.0) {
            if (threadIdx.x == 0) *status = SIE_ERR_BREAKDOWN;
            return;
        }
        for (int32_t cp = c + 1 + threadIdx.x; cp < pe; cp += blockDim.x) wc[cp - p] = F[int64_t(c) * nf + cp];
        __syncthreads();
        const double den = d.x * d.x + d.y * d.y;
        const double2 inv = make_double2(d.x / den, -d.y / den);
        for (int32_t i = c + 1 + threadIdx.x; i < nf; i += blockDim.x) {
            const double2 l = cmul(F[int64_t(c) * nf + i], inv);
            F[int64_t(c) * nf + i] = l;
            const int32_t last = min(pe - 1, i);
            for (int32_t cp = c + 1; cp <= last; ++cp)
                F[int64_t(cp) * nf + i] = csub(F[int64_t(cp) * nf + i], cmul(l, wc[cp - p]));
        }
    }
}

// Trailing update of the panel [p, pe): F_ij -= sum_c l_ic d_c l_jc for
// pe <= j <= i < nf, in 32 x 32 tiles of the lower triangle (blockIdx.y
// enumerates a front's tiles row by row).
__global__ void __launch_bounds__(256) k_nd_update(FrontArgs fa, int32_t lvl0, int32_t p, double2 *__restrict__ W) {
    const int32_t f = fa.order[lvl0 + blockIdx.x];
    const int32_t nf = fa.nf[f], nv = fa.nv[f];
    if (nv <= p) return;
    const int32_t pe = min(p + kPanel, nv), pw = pe - p;
    const int32_t ns = nf - pe;
    if (ns <= 0) return;
    const int32_t nt = (ns + kTile - 1) / kTile;
    const int64_t k = blockIdx.y;
    if (k >= int64_t(nt) * (nt + 1) / 2) return;
    int32_t ti = int32_t((sqrt(8.0 * double(k) + 1.0) - 1.0) * 0.5);
    while (int64_t(ti) * (ti + 1) / 2 > k) --ti;
    while (int64_t(ti + 1) * (ti + 2) / 2 <= k) ++ti;
    const int32_t tj = int32_t(k - int64_t(ti) * (ti + 1) / 2);
    const int32_t r0 = pe + ti * kTile, c0 = pe + tj * kTile;
    const double2 *Fc = W + fa.Foff[f];
    double2 *F = W + fa.Foff[f];
    __shared__ double2 A[kPanel][kTile + 1], B[kPanel][kTile + 1];   // A[c][row], B[c][col] (times d_c)
    for (int t = threadIdx.x; t < kPanel * kTile; t += blockDim.x) {
        const int c = t / kTile, x = t % kTile;
        double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
        if (c < pw) {
            const int64_t col = int64_t(p + c) * nf;
            if (r0 + x < nf) va = Fc[col + r0 + x];
            if (c0 + x < nf) vb = cmul(Fc[col + c0 + x], Fc[col + p + c]);
        }
        A[c][x] = va;
        B[c][x] = vb;
    }
    __syncthreads();
    const int x = threadIdx.x % kTile, yq = threadIdx.x / kTile;   // row x, columns yq + 8 q
    double2 acc[4];
    for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int c = 0; c < pw; ++c) {
        const double2 av = A[c][x];
        for (int q = 0; q < 4; ++q) {
            const double2 bv = B[c][yq + 8 * q];
            acc[q].x += av.x * bv.x - av.y * bv.y;
            acc[q].y += av.x * bv.y + av.y * bv.x;
        }
    }
    const int32_t i = r0 + x;
    if (i >= nf) return;
    for (int q = 0; q < 4; ++q) {
        const int32_t j = c0 + yq + 8 * q;
        if (j < nf && j <= i) {
            double2 &dst = F[int64_t(j) * nf + i];
            dst = csub(dst, acc[q]);
        }
    }
}

// The factor of each front (its first nv columns) into the slot's storage,
// in FP64 and rounded to FP32.
__global__ void k_nd_store(FrontArgs fa, const double2 *__restrict__ W, double2 *__restrict__ L64,
                           float2 *__restrict__ L32) {
    const int32_t f = blockIdx.x;
    const int64_t n = int64_t(fa.nf[f]) * fa.nv[f];
    const double2 *F = W + fa.Foff[f];
    double2 *d = L64 + fa.Loff[f];
    float2 *e = L32 + fa.Loff[f];
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        const double2 v = F[t];
        d[t] = v;
        e[t] = make_float2(float(v.x), float(v.y));
    }
}

// ---------------------------------------------------------------- solve kernels

// Right-hand sides per solve CTA: a group of up to kG right-hand sides that
// share a factor slot (the ports of one frequency), so that a front's factor
// is read once for all of them.
constexpr int kG = 4;

// Forward: per (front, group of right-hand sides) the frontal vectors
// v = [rhs(I_f); 0] plus the children's update vectors, the unit lower L_11
// solve on the pivots, v_U -= L_21 z_I, z_I back into u and v_U to the update
// vector of f.  Pivots go 32 at a time: the chunk's 32 x 32 block is staged in
// shared memory, warp 0 solves it in registers (a shuffle hands each pivot to
// the lanes below it), then every thread applies the chunk's 32 columns to one
// of the rows below: three barriers per 32 pivots.  u: [R][nunk]; uv:
// [R][sumU]; grp: [ngroups][kG] right-hand sides (-1: none), all of one slot;
// v in shared memory: [kG][ldv].
template <typename T>
__global__ void __launch_bounds__(256) k_nd_fwd(FrontArgs fa, int32_t lvl0, const C<T> *__restrict__ L, int64_t sumL,
                                                const int32_t *__restrict__ grp, const int32_t *__restrict__ slot,
                                                int64_t nunk, int64_t sumU, int32_t ldv, C<T> *__restrict__ u,
                                                C<T> *__restrict__ uv) {
    extern __shared__ __align__(16) unsigned char nd_smem[];
    C<T> *v = reinterpret_cast<C<T> *>(nd_smem);
    __shared__ C<T> blk[32][33];   // blk[j][l] = L[c0 + l][c0 + j]: the chunk's block, column j
    const int32_t f = fa.order[lvl0 + blockIdx.x];
    const int32_t *gr = grp + int64_t(blockIdx.y) * kG;
    const int32_t nf = fa.nf[f], nv = fa.nv[f];
    const C<T> *Lf = L + int64_t(slot[gr[0]]) * sumL + fa.Loff[f];
    const int lane = threadIdx.x & 31;
    const C<T> zero = mk<T>(T(0), T(0));
    for (int g = 0; g < kG; ++g) {
        const int32_t r = gr[g];
        const C<T> *ur = u + int64_t(r < 0 ? 0 : r) * nunk + fa.first[f];
        for (int32_t t = threadIdx.x; t < nf; t += blockDim.x) v[g * ldv + t] = (r >= 0 && t < nv) ? ur[t] : zero;
    }
    for (int32_t q = fa.child_ptr[f]; q < fa.child_ptr[f + 1]; ++q) {
        __syncthreads();
        const int32_t c = fa.child[q];
        const int32_t mc = fa.nf[c] - fa.nv[c];
        const int32_t *rp = fa.relpos + fa.Uoff[c];
        for (int g = 0; g < kG; ++g) {
            const int32_t r = gr[g];
            if (r < 0) continue;
            const C<T> *uc = uv + int64_t(r) * sumU + fa.Uoff[c];
            for (int32_t t = threadIdx.x; t < mc; t += blockDim.x) v[g * ldv + rp[t]] = cadd(v[g * ldv + rp[t]], uc[t]);
        }
    }
    for (int32_t c0 = 0; c0 < nv; c0 += 32) {
        const int32_t cw = min(32, nv - c0);
        __syncthreads();
        for (int32_t t = threadIdx.x; t < 32 * 32; t += blockDim.x) {   // stage the block (coalesced)
            const int32_t c = t >> 5, rr = t & 31;
            blk[c][rr] = (rr < cw && c < cw) ? Lf[int64_t(c0 + c) * nf + c0 + rr] : zero;
        }
        __syncthreads();
        if (threadIdx.x < 32) {   // the chunk's diagonal block, lane l on pivot row c0 + l
            C<T> vl[kG];
#pragma unroll
            for (int g = 0; g < kG; ++g) vl[g] = lane < cw ? v[g * ldv + c0 + lane] : zero;
            for (int32_t j = 0; j < cw; ++j) {
                const C<T> l = blk[j][lane];
#pragma unroll
                for (int g = 0; g < kG; ++g) {
                    C<T> y;
                    y.x = __shfl_sync(0xffffffffu, vl[g].x, j);
                    y.y = __shfl_sync(0xffffffffu, vl[g].y, j);
                    if (lane > j) vl[g] = csub(vl[g], cmul(l, y));
                }
            }
            if (lane < cw)
#pragma unroll
                for (int g = 0; g < kG; ++g) v[g * ldv + c0 + lane] = vl[g];
        }
        __syncthreads();
        for (int32_t i = c0 + cw + threadIdx.x; i < nf; i += blockDim.x) {   // rows below the chunk
            C<T> acc[kG];
#pragma unroll
            for (int g = 0; g < kG; ++g) acc[g] = zero;
#pragma unroll 4
            for (int32_t j = 0; j < cw; ++j) {
                const C<T> l = Lf[int64_t(c0 + j) * nf + i];
#pragma unroll
                for (int g = 0; g < kG; ++g) acc[g] = cadd(acc[g], cmul(l, v[g * ldv + c0 + j]));
            }
#pragma unroll
            for (int g = 0; g < kG; ++g) v[g * ldv + i] = csub(v[g * ldv + i], acc[g]);
        }
    }
    __syncthreads();
    for (int g = 0; g < kG; ++g) {
        const int32_t r = gr[g];
        if (r < 0) continue;
        C<T> *ur = u + int64_t(r) * nunk + fa.first[f];
        C<T> *uvr = uv + int64_t(r) * sumU + fa.Uoff[f];
        for (int32_t t = threadIdx.x; t < nf; t += blockDim.x) {
            if (t < nv) ur[t] = v[g * ldv + t];
            else uvr[t - nv] = v[g * ldv + t];
        }
    }
}

template <typename V> __device__ __forceinline__ V warp_sum(V a) {
    for (int s = 16; s > 0; s >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, s);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, s);
    }
    return a;
}

// Backward: per (front, group of right-hand sides) w_I = z_I / d - L_21^T x(U_f),
// then L_11^T x_I = w_I from the last pivot down, 32 pivots at a time: first
// the pivots after the chunk, already solved, enter by column dot products (one
// warp per chunk column, coalesced), then warp 0 solves the chunk's
// upper-triangular block (staged in shared memory) with shuffles.  x_I back
// into u.
template <typename T>
__global__ void __launch_bounds__(256) k_nd_bwd(FrontArgs fa, int32_t lvl0, const C<T> *__restrict__ L, int64_t sumL,
                                                const int32_t *__restrict__ grp, const int32_t *__restrict__ slot,
                                                int64_t nunk, int32_t ldv, C<T> *__restrict__ u) {
    extern __shared__ __align__(16) unsigned char nd_smem[];
    C<T> *v = reinterpret_cast<C<T> *>(nd_smem);   // [kG][ldv]: x_I (pivots), then x(U_f)
    __shared__ C<T> blk[32][33];                   // blk[j][l] = L[c0 + j][c0 + l]
    const int32_t f = fa.order[lvl0 + blockIdx.x];
    const int32_t *gr = grp + int64_t(blockIdx.y) * kG;
    const int32_t nf = fa.nf[f], nv = fa.nv[f];
    if (nv == 0) return;
    const C<T> *Lf = L + int64_t(slot[gr[0]]) * sumL + fa.Loff[f];
    const int32_t *ui = fa.uidx + fa.Uoff[f];
    const C<T> zero = mk<T>(T(0), T(0));
    for (int g = 0; g < kG; ++g) {
        const int32_t r = gr[g];
        const C<T> *ubase = u + int64_t(r < 0 ? 0 : r) * nunk;
        const C<T> *ur = ubase + fa.first[f];
        for (int32_t t = threadIdx.x; t < nf; t += blockDim.x) {
            C<T> val = zero;
            if (r >= 0) {
                if (t < nv) {
                    const C<T> d = Lf[int64_t(t) * nf + t];
                    const T den = d.x * d.x + d.y * d.y;
                    val = cmul(ur[t], mk<T>(d.x / den, -d.y / den));
                } else {
                    val = ubase[ui[t - nv]];
                }
            }
            v[g * ldv + t] = val;
        }
    }
    __syncthreads();
    // w_I -= L_21^T x_U: one warp per pivot column
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int32_t li = wid; li < nv; li += nw) {
        const C<T> *col = Lf + int64_t(li) * nf;
        C<T> acc[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) acc[g] = zero;
        for (int32_t t = nv + lane; t < nf; t += 32) {
            const C<T> l = col[t];
#pragma unroll
            for (int g = 0; g < kG; ++g) acc[g] = cadd(acc[g], cmul(l, v[g * ldv + t]));
        }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            acc[g] = warp_sum(acc[g]);
            if (lane == 0) v[g * ldv + li] = csub(v[g * ldv + li], acc[g]);
        }
    }
    for (int32_t c0 = ((nv - 1) / 32) * 32; c0 >= 0; c0 -= 32) {
        const int32_t cw = min(32, nv - c0), ce = c0 + cw;
        __syncthreads();
        // the solved pivots ce .. nv-1 into the chunk's rows: x_j -= sum_{i >= ce} l_ij x_i
        for (int32_t jj = wid; jj < cw; jj += nw) {
            const C<T> *col = Lf + int64_t(c0 + jj) * nf;
            C<T> acc[kG];
#pragma unroll
            for (int g = 0; g < kG; ++g) acc[g] = zero;
            for (int32_t i = ce + lane; i < nv; i += 32) {
                const C<T> l = col[i];
#pragma unroll
                for (int g = 0; g < kG; ++g) acc[g] = cadd(acc[g], cmul(l, v[g * ldv + i]));
            }
#pragma unroll
            for (int g = 0; g < kG; ++g) {
                acc[g] = warp_sum(acc[g]);
                if (lane == 0) v[g * ldv + c0 + jj] = csub(v[g * ldv + c0 + jj], acc[g]);
            }
        }
        // the chunk's block of L (rows and columns c0 .. ce-1), staged for the lanes' row reads
        for (int32_t t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
            const int32_t c = t >> 5, rr = t & 31;   // column c0 + c, row c0 + rr
            blk[rr][c] = (rr < cw && c < cw) ? Lf[int64_t(c0 + c) * nf + c0 + rr] : zero;
        }
        __syncthreads();
        if (threadIdx.x < 32) {   // upper-triangular block, lane l on pivot c0 + l, last pivot first
            C<T> xl[kG];
#pragma unroll
            for (int g = 0; g < kG; ++g) xl[g] = lane < cw ? v[g * ldv + c0 + lane] : zero;
            for (int32_t j = cw - 1; j >= 0; --j) {
                const C<T> l = blk[j][lane];
#pragma unroll
                for (int g = 0; g < kG; ++g) {
                    C<T> x;
                    x.x = __shfl_sync(0xffffffffu, xl[g].x, j);
                    x.y = __shfl_sync(0xffffffffu, xl[g].y, j);
                    if (lane < j) xl[g] = csub(xl[g], cmul(l, x));
                }
            }
            if (lane < cw)
#pragma unroll
                for (int g = 0; g < kG; ++g) v[g * ldv + c0 + lane] = xl[g];
        }
    }
    __syncthreads();
    for (int g = 0; g < kG; ++g) {
        const int32_t r = gr[g];
        if (r < 0) continue;
        C<T> *ur = u + int64_t(r) * nunk + fa.first[f];
        for (int32_t t = threadIdx.x; t < nv; t += blockDim.x) ur[t] = v[g * ldv + t];
    }
}

}  // namespace

// Builds the ordering and the symbolic factorisation.  uadj: adjacency of the
// nunk unknowns (raw numbering); xyz: [nunk][3] positions.  perm (new -> raw)
// is returned; the state's row data come later from nd_rows.
int nd_build(const std::vector<std::vector<int32_t>> &uadj, const std::vector<double> &xyz, std::vector<int32_t> &perm,
             NdState **out) {
    const int64_t nunk = int64_t(uadj.size());
    auto *s = new (std::nothrow) NdState;
    if (!s) return fail(SIE_ERR_OOM, "preconditioner: out of host memory");
    *out = s;
    s->nunk = nunk;
    std::vector<Node> tree;
    perm.clear();
    perm.reserve(nunk);
    Dissect ds{uadj, xyz, perm, tree, std::vector<int8_t>(nunk, 0)};
    std::vector<int32_t> all(nunk);
    std::iota(all.begin(), all.end(), 0);
    ds.rec(std::move(all));
    std::vector<int32_t> inv(nunk);
    for (int64_t i = 0; i < nunk; ++i) inv[perm[i]] = int32_t(i);
    const int32_t F = int32_t(tree.size());
    s->nfront = F;
    // update sets U_f in postorder (the tree's creation order)
    std::vector<std::vector<int32_t>> U(F);
    std::vector<int32_t> parent(F, -1);
    for (int32_t f = 0; f < F; ++f)
        for (int32_t c : tree[f].children) parent[c] = f;
    for (int32_t f = 0; f < F; ++f) {
        const int64_t end = tree[f].first + tree[f].nv;
        std::vector<int32_t> cand;
        for (int64_t i = tree[f].first; i < end; ++i)
            for (int32_t w : uadj[perm[i]])
                if (inv[w] >= end) cand.push_back(inv[w]);
        for (int32_t c : tree[f].children)
            for (int32_t j : U[c])
                if (j >= end) cand.push_back(j);
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        U[f] = std::move(cand);
    }
    // levels by height, offsets
    std::vector<int32_t> height(F, 0);
    int32_t H = 0;
    for (int32_t f = 0; f < F; ++f) {
        for (int32_t c : tree[f].children) height[f] = std::max(height[f], height[c] + 1);
        H = std::max(H, height[f]);
    }
    std::vector<int64_t> first(F), Foff(F), Loff(F), Uoff(F);
    std::vector<int32_t> nv(F), nf(F), child_ptr(F + 1, 0), child, uidx, relpos;
    int64_t sF = 0, sL = 0, sU = 0;
    for (int32_t f = 0; f < F; ++f) {
        first[f] = tree[f].first;
        nv[f] = tree[f].nv;
        nf[f] = tree[f].nv + int32_t(U[f].size());
        Foff[f] = sF;
        Loff[f] = sL;
        Uoff[f] = sU;
        sF += int64_t(nf[f]) * nf[f];
        sL += int64_t(nf[f]) * nv[f];
        sU += int64_t(U[f].size());
        s->max_nf = std::max(s->max_nf, nf[f]);
        const double a = nv[f], m = double(U[f].size());
        s->flops += int64_t(a * a * a / 3.0 + a * a * m + a * m * m);
        for (int32_t c : tree[f].children) child.push_back(c);
        child_ptr[f + 1] = int32_t(child.size());
    }
    s->sumF = sF;
    s->sumL = sL;
    s->sumU = sU;
    uidx.resize(sU);
    relpos.assign(sU, 0);
    for (int32_t f = 0; f < F; ++f) std::copy(U[f].begin(), U[f].end(), uidx.begin() + Uoff[f]);
    for (int32_t c = 0; c < F; ++c) {
        const int32_t f = parent[c];
        if (f < 0) continue;
        const int64_t end = first[f] + nv[f];
        for (size_t a = 0; a < U[c].size(); ++a) {
            const int32_t j = U[c][a];
            relpos[Uoff[c] + a] = j < end ? int32_t(j - first[f])
                                          : nv[f] + int32_t(std::lower_bound(U[f].begin(), U[f].end(), j) - U[f].begin());
        }
    }
    std::vector<int32_t> order;
    s->level_ptr.assign(1, 0);
    for (int32_t h = 0; h <= H; ++h) {
        int32_t mnv = 0, mnf = 0;
        for (int32_t f = 0; f < F; ++f)
            if (height[f] == h) {
                order.push_back(f);
                mnv = std::max(mnv, nv[f]);
                mnf = std::max(mnf, nf[f]);
            }
        s->level_ptr.push_back(int32_t(order.size()));
        s->level_max_nv.push_back(mnv);
        s->level_max_nf.push_back(mnf);
    }
    int rc;
    if ((rc = nd_upload(s, &s->order, order))) return rc;
    if ((rc = nd_upload(s, &s->first, first))) return rc;
    if ((rc = nd_upload(s, &s->Foff, Foff))) return rc;
    if ((rc = nd_upload(s, &s->Loff, Loff))) return rc;
    if ((rc = nd_upload(s, &s->Uoff, Uoff))) return rc;
    if ((rc = nd_upload(s, &s->nv, nv))) return rc;
    if ((rc = nd_upload(s, &s->nf, nf))) return rc;
    if ((rc = nd_upload(s, &s->child_ptr, child_ptr))) return rc;
    if ((rc = nd_upload(s, &s->child, child))) return rc;
    if ((rc = nd_upload(s, &s->uidx, uidx))) return rc;
    if ((rc = nd_upload(s, &s->relpos, relpos))) return rc;
    return SIE_OK;
}

// Positions of the Laplacian's row entries in their fronts: for pivot i of
// front f and the entry to unknown j (row_oth, new numbering, -1 for a fixed
// node or the same unknown): j - first_f for a later pivot of f (lower
// triangle), nv_f + (position of j in U_f) for j in U_f, -1 otherwise (an
// earlier pivot of f, whose own row adds the entry, or an unknown of an
// earlier front, whose front added it).
int nd_rows(NdState *s, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &row_oth) {
    const int32_t F = s->nfront;
    std::vector<int64_t> first(F), Uoff(F);
    std::vector<int32_t> nv(F), nf(F);
    SIE_CUDA(cudaMemcpy(first.data(), s->first, F * sizeof(int64_t), cudaMemcpyDeviceToHost));
    SIE_CUDA(cudaMemcpy(Uoff.data(), s->Uoff, F * sizeof(int64_t), cudaMemcpyDeviceToHost));
    SIE_CUDA(cudaMemcpy(nv.data(), s->nv, F * sizeof(int32_t), cudaMemcpyDeviceToHost));
    SIE_CUDA(cudaMemcpy(nf.data(), s->nf, F * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int32_t> uidx(std::max<int64_t>(s->sumU, 1));
    if (s->sumU) SIE_CUDA(cudaMemcpy(uidx.data(), s->uidx, s->sumU * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int32_t> front_of(s->nunk, -1);
    for (int32_t f = 0; f < F; ++f)
        for (int32_t k = 0; k < nv[f]; ++k) front_of[first[f] + k] = f;
    std::vector<int32_t> loc(row_oth.size(), -1);
    for (int64_t i = 0; i < s->nunk; ++i) {
        const int32_t f = front_of[i];
        const int64_t end = first[f] + nv[f];
        const int32_t *Ub = uidx.data() + Uoff[f], *Ue = Ub + (nf[f] - nv[f]);
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const int32_t j = row_oth[k];
            if (j < 0 || j == i) continue;
            if (j > i && j < end) loc[k] = int32_t(j - first[f]);
            else if (j >= end) {
                const int32_t *q = std::lower_bound(Ub, Ue, j);
                if (q == Ue || *q != j) return fail(SIE_ERR_ARG, "preconditioner: nested dissection lost a coupling");
                loc[k] = nv[f] + int32_t(q - Ub);
            }
        }
    }
    return nd_upload(s, &s->row_loc, loc);
}

int64_t nd_factor_size(const NdState *s) { return s->sumL; }
int64_t nd_workspace_size(const NdState *s) { return s->sumF; }
int64_t nd_update_size(const NdState *s) { return s->sumU; }
void nd_info(const NdState *s, int32_t *fronts, int64_t *nnz, int32_t *max_front, int64_t *flops) {
    if (fronts) *fronts = s->nfront;
    if (nnz) *nnz = s->sumL;
    if (max_front) *max_front = s->max_nf;
    if (flops) *flops = s->flops;
}

static FrontArgs front_args(const NdState *s) {
    return FrontArgs{s->order, s->first, s->Foff, s->Loff, s->Uoff, s->nv, s->nf, s->child_ptr, s->child, s->uidx,
                     s->relpos};
}

// LDL^T of one frequency slot: a = admittances [nb] of the slot, W the front
// workspace [sumF], the factor into L64 / L32 [sumL].
int nd_factor(pfft_plan *p, NdState *s, const double2 *a, const int32_t *row_ptr, const int32_t *row_br,
              double2 *W, double2 *L64, float2 *L32, int *status, cudaStream_t st) {
    const FrontArgs fa = front_args(s);
    const int32_t H = int32_t(s->level_ptr.size()) - 1;
    for (int32_t h = 0; h < H; ++h) {
        const int32_t l0 = s->level_ptr[h], nfr = s->level_ptr[h + 1] - l0;
        if (nfr == 0) continue;
        k_nd_assemble<<<nfr, 256, 0, st>>>(fa, l0, a, row_ptr, row_br, s->row_loc, W);
        SIE_LAUNCH_CHECK(p);
        for (int32_t pp = 0; pp < s->level_max_nv[h]; pp += kPanel) {
            k_nd_panel<<<nfr, 256, 0, st>>>(fa, l0, pp, W, status);
            SIE_LAUNCH_CHECK(p);
            // widest trailing part of any front of the level: nf - pe with pe >= pp + 1
            const int32_t ns = s->level_max_nf[h] - (pp + 1);
            if (ns <= 0) continue;
            const int64_t nt = (ns + kTile - 1) / kTile;
            const int64_t tiles = nt * (nt + 1) / 2;
            if (tiles > 65535) return fail(SIE_ERR_ARG, "preconditioner: nested-dissection front too large");
            k_nd_update<<<dim3(unsigned(nfr), unsigned(tiles)), 256, 0, st>>>(fa, l0, pp, W);
            SIE_LAUNCH_CHECK(p);
        }
    }
    k_nd_store<<<s->nfront, 256, 0, st>>>(fa, W, L64, L32);
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

// z = K^-1 rhs in place on u [R][nunk] (new numbering) with the factors of each
// right-hand side's slot (L [nslots][sumL]); grp: [ngrp][kG] groups of right-hand
// sides sharing a slot (-1 pads); uv: update vectors [R][sumU].
template <typename T>
int nd_solve(pfft_plan *p, const NdState *s, const C<T> *L, const int32_t *slot, const int32_t *grp, int32_t ngrp,
             C<T> *u, C<T> *uv, cudaStream_t st) {
    const FrontArgs fa = front_args(s);
    const int32_t H = int32_t(s->level_ptr.size()) - 1;
    const size_t smax = size_t(kG) * std::max(s->max_nf, 1) * sizeof(C<T>);
    if (smax > 180 * 1024)
        return fail(SIE_ERR_ARG, "preconditioner: a nested-dissection front of " + std::to_string(s->max_nf) +
                                     " unknowns exceeds the solve's shared memory");
    if (int rc = set_smem((const void *)k_nd_fwd<T>, smax)) return rc;
    if (int rc = set_smem((const void *)k_nd_bwd<T>, smax)) return rc;
    // each level's frontal vectors sized by its own largest front (the leaves are small:
    // more CTAs resident per SM)
    for (int32_t h = 0; h < H; ++h) {
        const int32_t l0 = s->level_ptr[h], nfr = s->level_ptr[h + 1] - l0;
        if (!nfr) continue;
        const int32_t ldv = std::max(s->level_max_nf[h], 1);
        const size_t sm = size_t(kG) * ldv * sizeof(C<T>);
        k_nd_fwd<T><<<dim3(unsigned(nfr), unsigned(ngrp)), 256, sm, st>>>(fa, l0, L, s->sumL, grp, slot, s->nunk,
                                                                           s->sumU, ldv, u, uv);
        SIE_LAUNCH_CHECK(p);
    }
    for (int32_t h = H - 1; h >= 0; --h) {
        const int32_t l0 = s->level_ptr[h], nfr = s->level_ptr[h + 1] - l0;
        if (!nfr) continue;
        const int32_t ldv = std::max(s->level_max_nf[h], 1);
        const size_t sm = size_t(kG) * ldv * sizeof(C<T>);
        k_nd_bwd<T><<<dim3(unsigned(nfr), unsigned(ngrp)), 256, sm, st>>>(fa, l0, L, s->sumL, grp, slot, s->nunk,
                                                                           ldv, u);
        SIE_LAUNCH_CHECK(p);
    }
    return SIE_OK;
}
template int nd_solve<double>(pfft_plan *, const NdState *, const double2 *, const int32_t *, const int32_t *,
                              int32_t, double2 *, double2 *, cudaStream_t);
template int nd_solve<float>(pfft_plan *, const NdState *, const float2 *, const int32_t *, const int32_t *, int32_t,
                             float2 *, float2 *, cudaStream_t);
int nd_group_size() { return kG; }

void nd_free(NdState *s) {
    if (!s) return;
    for (void *a : s->allocs) cudaFree(a);
    delete s;
}

}  // namespace sie
