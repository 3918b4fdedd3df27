// Pre-corrected near field on the tensor cores (Sec. IV-B step 4, Eq. Lb) for
// the mixed form, fused with the per-triangle output y_T (Eq. Zb).
//
// The near matrix L_d is block-sparse with 3x3 real blocks.  Rows are cut
// into tiles of 42 consecutive triangles (126 rows of the M = 128 MMA tile,
// row m = 3 t_local + k).  A tile's columns are the union U of the near
// triangles of its rows, ascending; each column triangle T' contributes 4
// K-slots (its local currents l = 0, 1, 2 and a zero), so one
// M = 128, N = 256, K = 8 step covers two column triangles, and a pipeline
// chunk four (two K steps: the per-chunk waits, fences, arrivals and copy
// issues of the feed are shared by twice the work of one step).  N = 256 real
// columns are 128 complex right-hand sides (column 2r the real part, 2r + 1
// the imaginary part): L_d is real, so real and imaginary parts are
// independent columns of one real product.
//
// Precision (kind::tf32 with split operands): every operand v is split on chip
// into v_b + v_s, v_b the tf32 rounding of v and v_s = v - v_b, and the
// product is accumulated in fp32 as A_b X_b + A_b X_s + A_s X_b (the dropped
// A_s X_s and the tf32 reading of v_s are below 2^-21 relative per product).
//
// Data in device memory, fp32 and compact: the A operand (dense near blocks
// of each tile) [union position][128 rows][3] (1.5 KB per position, built at
// plan creation), the B operand read straight from c_T [T][3][R] (three 1 KB
// rows per triangle and slab of 128 right-hand sides).
//
// Persistent CTAs (one per SM) walk the (tile, slab) items; warp roles:
//   warp 0     producer: bulk copies of the compact operands, 4-stage raw ring
//   warp 1     TMEM owner (2 accumulators x 256 columns) and MMA issuer
//   warps 2-5  converters: raw ring -> split, MMA-layout images (2-stage ring)
//   warps 6-9  epilogue: accumulator -> + far field + Z_s Gram term -> y_T
//              (double-float complex), overlapping the next item's MMAs
//              (double-buffered TMEM)
// Every wait is bounded (2 s); a wait that runs out sets the plan's error
// flag, the role stops, and the CTA still drains its MMAs and frees its TMEM.
#include <algorithm>
#include <cstring>
#include <vector>

#include "sie_dd.cuh"
#include "sie_plan.h"
#include "sie_tc.cuh"

using namespace sie;

namespace {

constexpr int kTileTri = 42;                    // triangles per row tile
constexpr int kRows = 128;                      // MMA M
constexpr int kCols = 256;                      // MMA N (128 complex right-hand sides)
constexpr int kSlabRhs = kCols / 2;
constexpr int kPos = 4;                        // column triangles per chunk: two K = 8 steps
constexpr int kRawStages = 4, kCvStages = 2;
constexpr uint32_t kARaw = kRows * 3 * 4;       // compact A bytes per union position (1.5 KB)
constexpr uint32_t kXRow = kSlabRhs * 8;        // one c_T row of a slab (1 KB)
constexpr uint32_t kRawBytes = kPos * kARaw + kPos * 3 * kXRow;    // 18 KB
constexpr uint32_t kAImg = kRows * 16;          // A image per position (2 KB)
constexpr uint32_t kXImg = kCols * 16;          // X image per triangle (4 KB)
constexpr uint32_t kCvBytes = 2 * (kPos * kAImg) + 2 * (kPos * kXImg);  // 48 KB
constexpr uint32_t kSmemBytes = kRawStages * kRawBytes + kCvStages * kCvBytes + 1024;
constexpr int kThreads = 320;
constexpr uint64_t kWaitNs = 2000000000ull;     // bounded mbarrier waits: 2 s
constexpr uint32_t kErrNearMma = 1;

struct NearMmaArgs {
    const int64_t *u_ptr;     // [ntiles + 1], counts multiples of kPos
    const int32_t *u_tri;     // [n_union]
    const float *Ac;          // [n_union][128][3]
    const float2 *ffar;       // [nt][3][R]
    const float2 *cT;         // [nt][3][R]
    const double *gram;       // [nt][3][3]
    const int32_t *cond;      // [nt]
    const float2 *coef;       // [R][2 ncond + 1] double-float (hi, lo)
    int ncond;
    int64_t nt;
    int32_t R;                // even
    int32_t ntiles, nslab;
    float4 *y_tri;            // [R][nt][3] double-float complex
    int *err;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void split4(float a0, float a1, float a2, float4 &b, float4 &s) {
    const float b0 = tc::round_tf32(a0), b1 = tc::round_tf32(a1), b2 = tc::round_tf32(a2);
    b = make_float4(b0, b1, b2, 0.f);
    s = make_float4(a0 - b0, a1 - b1, a2 - b2, 0.f);
}

__global__ void __launch_bounds__(kThreads, 1) k_near_mma(NearMmaArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t raw_full[kRawStages], raw_empty[kRawStages];
    __shared__ __align__(8) uint64_t cv_full[kCvStages], cv_empty[kCvStages];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drained;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *base = smem_raw + ((1024 - (tc::smem_u32(smem_raw) & 1023)) & 1023);
    unsigned char *raw = base;                                  // [kRawStages][kRawBytes]
    unsigned char *cv = base + kRawStages * kRawBytes;          // [kCvStages][kCvBytes]
    const int nitems = a.ntiles * a.nslab;
    const int32_t R = a.R;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRawStages; ++s) { tc::mbar_init(&raw_full[s], 1); tc::mbar_init(&raw_empty[s], 128); }
        for (int s = 0; s < kCvStages; ++s) { tc::mbar_init(&cv_full[s], 128); tc::mbar_init(&cv_empty[s], 1); }
        for (int s = 0; s < 2; ++s) { tc::mbar_init(&acc_full[s], 1); tc::mbar_init(&acc_empty[s], 128); }
        tc::mbar_init(&drained, 1);
        tc::mbar_fence_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_slot, 2 * kCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ---- producer: compact A of two positions + c_T rows of two triangles per chunk
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
                const int tile = w % a.ntiles, slab = w / a.ntiles;
                const int64_t u0 = a.u_ptr[tile];
                const int nchunk = int((a.u_ptr[tile + 1] - u0) / kPos);
                const int32_t nr = min(kSlabRhs, R - slab * kSlabRhs);
                const uint32_t xbytes = uint32_t(nr) * 8;
                for (int c = 0; c < nchunk; ++c, ++g) {
                    const uint32_t s = g % kRawStages, use = g / kRawStages;
                    if (use > 0 && !tc::mbar_wait(&raw_empty[s], (use - 1) & 1, kWaitNs)) { ok = false; break; }
                    unsigned char *st = raw + s * kRawBytes;
                    const int64_t u = u0 + kPos * c;
                    tc::mbar_expect_tx(&raw_full[s], kPos * kARaw + kPos * 3 * xbytes);
                    tc::bulk_g2s(st, a.Ac + u * (kARaw / 4), kPos * kARaw, &raw_full[s]);
                    for (int j = 0; j < kPos; ++j) {
                        const int64_t t = a.u_tri[u + j];
                        const float2 *src = a.cT + t * 3 * R + int64_t(slab) * kSlabRhs;
                        if (R == kSlabRhs) {   // the triangle's three rows are one contiguous 3 KB block
                            tc::bulk_g2s(st + kPos * kARaw + 3 * j * kXRow, src, 3 * kXRow, &raw_full[s]);
                        } else {
                            for (int l = 0; l < 3; ++l)
                                tc::bulk_g2s(st + kPos * kARaw + (3 * j + l) * kXRow, src + l * R, xbytes,
                                             &raw_full[s]);
                        }
                    }
                }
            }
            if (!ok) atomicOr(a.err, kErrNearMma);
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_tf32(kRows, kCols);
            uint32_t g = 0, item = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x, ++item) {
                const int tile = w % a.ntiles;
                const int nchunk = int((a.u_ptr[tile + 1] - a.u_ptr[tile]) / kPos);
                const uint32_t ab = item & 1, use_a = item >> 1;
                if (use_a > 0 && !tc::mbar_wait(&acc_empty[ab], (use_a - 1) & 1, kWaitNs)) { ok = false; break; }
                tc::fence_after_sync();
                const uint32_t d = tmem + ab * kCols;
                for (int c = 0; c < nchunk; ++c, ++g) {
                    const uint32_t s = g % kCvStages, use = g / kCvStages;
                    if (!tc::mbar_wait(&cv_full[s], use & 1, kWaitNs)) { ok = false; break; }
                    tc::fence_after_sync();
                    unsigned char *st = cv + s * kCvBytes;
                    // A images: core matrices (8 rows x 4 slots) +128 B along M, +2 KB along K;
                    // X images: (8 columns x 4 slots) +128 B along N, +4 KB along K; step ks
                    // takes positions 2 ks and 2 ks + 1 of the chunk
#pragma unroll
                    for (int ks = 0; ks < kPos / 2; ++ks) {
                        unsigned char *a0 = st + 2 * ks * kAImg, *x0 = st + 2 * kPos * kAImg + 2 * ks * kXImg;
                        const uint64_t Ab = tc::sdesc(a0, kAImg, 128), As = tc::sdesc(a0 + kPos * kAImg, kAImg, 128);
                        const uint64_t Xb = tc::sdesc(x0, kXImg, 128), Xs = tc::sdesc(x0 + kPos * kXImg, kXImg, 128);
                        tc::mma_tf32(d, Ab, Xb, idesc, c > 0 || ks > 0);
                        tc::mma_tf32(d, Ab, Xs, idesc, true);
                        tc::mma_tf32(d, As, Xb, idesc, true);
                    }
                    tc::mma_commit(&cv_empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&acc_full[ab]);
            }
            if (!ok) atomicOr(a.err, kErrNearMma);
            tc::mma_commit(&drained);   // every MMA of this CTA completed
            if (!tc::mbar_wait(&drained, 0, kWaitNs)) atomicOr(a.err, kErrNearMma);
        }
    } else if (warp < 6) {
        // ---- converters: raw ring -> split images
        const int tid = threadIdx.x - 64;
        uint32_t g = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
            const int tile = w % a.ntiles;
            const int nchunk = int((a.u_ptr[tile + 1] - a.u_ptr[tile]) / kPos);
            for (int c = 0; c < nchunk; ++c, ++g) {
                const uint32_t sr = g % kRawStages, ur = g / kRawStages;
                const uint32_t sc = g % kCvStages, uc = g / kCvStages;
                if (!tc::mbar_wait(&raw_full[sr], ur & 1, kWaitNs)) { ok = false; break; }
                if (uc > 0 && !tc::mbar_wait(&cv_empty[sc], (uc - 1) & 1, kWaitNs)) { ok = false; break; }
                const float *rA = reinterpret_cast<const float *>(raw + sr * kRawBytes);
                const float *rX = rA + kPos * kARaw / 4;
                float4 *img = reinterpret_cast<float4 *>(cv + sc * kCvBytes);
                float4 *iAb = img, *iAs = img + kPos * kAImg / 16;
                float4 *iXb = img + 2 * kPos * kAImg / 16, *iXs = iXb + kPos * kXImg / 16;
#pragma unroll
                for (int j = 0; j < kPos; ++j) {   // A: row tid of position j; image (g = m/8) * 128 B + (m % 8) * 16 B
                    const float *r3 = rA + j * (kARaw / 4) + 3 * tid;
                    float4 b, sp;
                    split4(r3[0], r3[1], r3[2], b, sp);
                    const int o = j * (kAImg / 16) + tid;
                    iAb[o] = b;
                    iAs[o] = sp;
                }
#pragma unroll
                for (int j = 0; j < kPos; ++j)   // X: columns n = tid, tid + 128 of triangle j
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int n = tid + 128 * h;
                        const float *x = rX + j * 3 * (kXRow / 4) + n;
                        float4 b, sp;
                        split4(x[0], x[kXRow / 4], x[2 * (kXRow / 4)], b, sp);
                        const int o = j * (kXImg / 16) + n;
                        iXb[o] = b;
                        iXs[o] = sp;
                    }
                fence_async_smem();
                mbar_arrive(&cv_full[sc]);
                mbar_arrive(&raw_empty[sr]);
            }
        }
        if (!ok && tid == 0) atomicOr(a.err, kErrNearMma);
    } else {
        // ---- epilogue
        const int q = warp & 3;
        const int m = 32 * q + lane;
        const int tl = m / 3, k = m - 3 * (m / 3);
        const int ldc = 2 * a.ncond + 1;
        uint32_t item = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < nitems; w += gridDim.x, ++item) {
            const int tile = w % a.ntiles, slab = w / a.ntiles;
            const uint32_t ab = item & 1, use_a = item >> 1;
            if (!tc::mbar_wait(&acc_full[ab], use_a & 1, kWaitNs)) { ok = false; break; }
            tc::fence_after_sync();
            const int64_t t = int64_t(tile) * kTileTri + tl;
            const bool active = m < 3 * kTileTri && t < a.nt;
            float G[3] = {0.f, 0.f, 0.f};
            int cd = 0;
            if (active) {
#pragma unroll
                for (int l = 0; l < 3; ++l) G[l] = float(a.gram[9 * t + 3 * k + l]);
                cd = a.cond[t];
            }
            const int32_t r0 = slab * kSlabRhs;
            const int32_t nr = min(kSlabRhs, R - r0);
            const float2 *ff = a.ffar + (t * 3 + k) * R + r0;
            const float2 *c0p = a.cT + (t * 3) * R + r0;
            for (int cc = 0; cc < kCols; cc += 32) {
                float v[32];
                __syncwarp();
                tc::tmem_ld32(tmem + ab * kCols + (uint32_t(32 * q) << 16) + uint32_t(cc), v);
                if (!active) continue;
                const int i0 = cc / 2;   // first right-hand side of this column block
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    if (i0 + i >= nr) continue;   // nr even: pairs stay whole
                    const float4 f2 = *reinterpret_cast<const float4 *>(ff + i0 + i);
                    const float4 x0 = *reinterpret_cast<const float4 *>(c0p + i0 + i);
                    const float4 x1 = *reinterpret_cast<const float4 *>(c0p + R + i0 + i);
                    const float4 x2 = *reinterpret_cast<const float4 *>(c0p + 2 * R + i0 + i);
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int32_t r = r0 + i0 + i + e;
                        // near + far exactly, as a double-float
                        const DD fr = two_sum(v[2 * (i + e)], e ? f2.z : f2.x);
                        const DD fi = two_sum(v[2 * (i + e) + 1], e ? f2.w : f2.y);
                        const float gr = G[0] * (e ? x0.z : x0.x) + G[1] * (e ? x1.z : x1.x) + G[2] * (e ? x2.z : x2.x);
                        const float gi = G[0] * (e ? x0.w : x0.y) + G[1] * (e ? x1.w : x1.y) + G[2] * (e ? x2.w : x2.y);
                        const float2 *cf = a.coef + int64_t(r) * ldc;
                        // Z_s * gram + j c_L * (near + far), combined in double-float
                        a.y_tri[(int64_t(r) * a.nt + t) * 3 + k] =
                            dd_zb(cf[2 * cd], cf[2 * cd + 1], cf[2 * a.ncond], gr, gi, fr, fi);
                    }
                }
            }
            tc::fence_before_sync();
            mbar_arrive(&acc_empty[ab]);
        }
        if (!ok && m == 0) atomicOr(a.err, kErrNearMma);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::fence_after_sync();
        tc::tmem_free(tmem, 2 * kCols);
    }
}

// Dense near blocks of each tile, compact fp32 [u][128 rows][3]: thread per (u, m).
__global__ void k_build_near_tiles(const int32_t *__restrict__ u_tile, const int32_t *__restrict__ u_col,
                                   int64_t n_union, const int64_t *__restrict__ near_ptr,
                                   const int32_t *__restrict__ near_col, const double *__restrict__ Ld, int64_t nt,
                                   float *__restrict__ Ac) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_union * kRows) return;
    const int64_t u = i / kRows;
    const int m = int(i % kRows);
    const int tl = m / 3, k = m % 3;
    const int64_t t = int64_t(u_tile[u]) * kTileTri + tl;
    const int32_t col = u_col[u];   // -1: padding position
    float v[3] = {0.f, 0.f, 0.f};
    if (m < 3 * kTileTri && t < nt && col >= 0) {
        int64_t lo = near_ptr[t], hi = near_ptr[t + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (near_col[mid] < col) lo = mid + 1; else hi = mid;
        }
        if (lo < near_ptr[t + 1] && near_col[lo] == col)
            for (int l = 0; l < 3; ++l) v[l] = float(Ld[9 * lo + 3 * k + l]);
    }
    for (int l = 0; l < 3; ++l) Ac[3 * i + l] = v[l];
}

// Self-test of the failure-detection path: one mbarrier that expects an arrival
// nothing makes, waited on with the same bounded wait as the tensor-core kernel;
// the wait runs out after limit_ns and sets the same error bit.
__global__ void k_selftest_wait(uint64_t limit_ns, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, limit_ns)) atomicOr(err, kErrNearMma);
}

}  // namespace

extern "C" int sie_selftest_bounded_wait(pfft_plan *p, double limit_ms, void *cuda_stream) {
    if (!p || !(limit_ms > 0.0) || limit_ms > 1000.0)
        return sie::fail(SIE_ERR_ARG, "sie_selftest_bounded_wait: limit must be in (0, 1000] ms");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    (void)cudaGetLastError();
    k_selftest_wait<<<1, 32, 0, st>>>(uint64_t(limit_ms * 1e6), p->d_err);
    SIE_CUDA(cudaGetLastError());
    return sie::finish_call(p, st);
}

namespace sie {

int near_mma_prepare(pfft_plan *p, const std::vector<int64_t> &near_ptr, const std::vector<int32_t> &near_col,
                     cudaStream_t s) {
    const int64_t nt = p->nt;
    const int64_t ntiles = (nt + kTileTri - 1) / kTileTri;
    std::vector<int64_t> u_ptr(ntiles + 1, 0);
    std::vector<int32_t> u_tri, u_col, u_tile;
    std::vector<int32_t> cols;
    for (int64_t i = 0; i < ntiles; ++i) {
        cols.clear();
        const int64_t t1 = std::min<int64_t>(nt, (i + 1) * kTileTri);
        for (int64_t t = i * kTileTri; t < t1; ++t)
            cols.insert(cols.end(), near_col.begin() + near_ptr[t], near_col.begin() + near_ptr[t + 1]);
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        for (int32_t c : cols) {
            u_tri.push_back(c);
            u_col.push_back(c);
            u_tile.push_back(int32_t(i));
        }
        for (size_t k = cols.size(); k % kPos; ++k) {   // pad to whole chunks: zero blocks on a valid triangle
            u_tri.push_back(cols.back());
            u_col.push_back(-1);
            u_tile.push_back(int32_t(i));
        }
        u_ptr[i + 1] = int64_t(u_tri.size());
    }
    const int64_t n_union = int64_t(u_tri.size());
    p->nm_tiles = ntiles;
    p->nm_union = n_union;
    int rc;
    auto up = [&](void **dst, const void *src, size_t bytes) -> int {
        int r = plan_alloc(p, dst, bytes);
        if (r) return r;
        SIE_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        return SIE_OK;
    };
    if ((rc = up((void **)&p->d_nm_uptr, u_ptr.data(), u_ptr.size() * 8))) return rc;
    if ((rc = up((void **)&p->d_nm_utri, u_tri.data(), u_tri.size() * 4))) return rc;
    int32_t *d_ucol = nullptr, *d_utile = nullptr;
    if ((rc = up((void **)&d_ucol, u_col.data(), u_col.size() * 4))) return rc;
    if ((rc = up((void **)&d_utile, u_tile.data(), u_tile.size() * 4))) return rc;
    if ((rc = plan_alloc(p, (void **)&p->d_nm_A, size_t(n_union) * kARaw))) return rc;
    const int64_t n = n_union * kRows;
    k_build_near_tiles<<<unsigned((n + 255) / 256), 256, 0, s>>>(d_utile, d_ucol, n_union, p->d_near_ptr,
                                                                 p->d_near_col, p->d_Ld64, nt, p->d_nm_A);
    p->launches++;
    SIE_CUDA(cudaGetLastError());
    SIE_CUDA(cudaStreamSynchronize(s));
    plan_free(p, d_ucol);
    plan_free(p, d_utile);
    return SIE_OK;
}

int near_mma_launch(pfft_plan *p, int32_t R, cudaStream_t st) {
    if (R % 2) return fail(SIE_ERR_ARG, "tensor-core near field: the right-hand-side count must be even");
    if (int rc = set_smem((const void *)k_near_mma, kSmemBytes)) return rc;
    int dev = 0, nsm = 0;
    SIE_CUDA(cudaGetDevice(&dev));
    SIE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    Scratch &s = p->scr;
    const int32_t nslab = (R + kSlabRhs - 1) / kSlabRhs;
    NearMmaArgs a{p->d_nm_uptr, p->d_nm_utri, p->d_nm_A, (const float2 *)s.ffar, (const float2 *)s.cT,
                  p->d_gram, p->d_cond, coef_dd(p), p->ncond, p->nt, R, int32_t(p->nm_tiles), nslab,
                  (float4 *)s.y_tri, p->d_err};
    const int64_t items = p->nm_tiles * nslab;
    k_near_mma<<<unsigned(std::min<int64_t>(items, nsm)), kThreads, kSmemBytes, st>>>(a);
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

}  // namespace sie
