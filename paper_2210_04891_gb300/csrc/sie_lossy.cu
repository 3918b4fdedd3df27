// The lossy-conductor kernel exp(-jkR)/R inside the pFFT product
// (pfft_params.kernel = SIE_KERNEL_LOSSY).
//
// The paper states only the static Green's function (Eq. StaticGF); the lossy
// variant replaces it, in the inductive term of Eq. Zb and in all four steps
// of Sec. IV-B, by the interior kernel of the same MQS equations,
// k = (1 - j)/delta with delta = sqrt(2 / (w mu0 sigma)), in the e^{jwt}
// convention of Z_s (Eq. ImpedanceOp).  Everything that depends on the kernel
// depends on the frequency, so it is built per angular frequency w and cached
// in slots:
//   - the folded complex spectrum of the kernel on the padded grid (FP64 and
//     rounded to FP32), used by the (y, z) convolution stage per grid;
//   - the pre-corrected near blocks L_d,k = L_direct,k - (I H_k B)_near
//     (complex, FP64 and rounded to FP32), where
//       L_direct,k = L_direct (the static closed-form blocks of the plan)
//                  + int int f.f' (exp(-jkR) - 1)/R, by the product of the
//                    7-point Radon rule on both triangles (the remainder is
//                    bounded: it tends to -(1 + j)/delta as R -> 0);
//   - the branch self terms Lt_k[e][e] for the preconditioner's diagonal.
// The right-hand sides of one call may have different frequencies: each grid
// of the convolution and each lane of the near-field gather looks up its own
// slot through small device tables (slot per right-hand side, per grid, and
// the slots' data pointers).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sie_plan.h"

namespace sie {

namespace {
constexpr int kLossyMaxSlots = 64;   // frequencies cached per plan
constexpr double kMu0 = 4e-7 * M_PI;
}  // namespace

struct LossySlot {
    double omega = -1.0;          // < 0: empty
    uint64_t last_use = 0;
    double2 *H64 = nullptr;       // folded spectrum [Mx/2+1][My/2+1][Mz/2+1], scaled by 1/(Mx My Mz)
    float2 *H32 = nullptr;
    double2 *Ld64 = nullptr;      // [n_near][3][3] L_direct,k - (I H_k B)
    float2 *Ld32 = nullptr;
    double2 *diagL = nullptr;     // [nb] Lt_k[e][e]
};

struct LossyCache {
    LossySlot slot[kLossyMaxSlots];
    uint64_t tick = 0;
    // device tables: per slot the data pointers (FP64 / FP32 spectra and near blocks)
    const void **d_htab64 = nullptr, **d_htab32 = nullptr, **d_ltab64 = nullptr, **d_ltab32 = nullptr;
    // per right-hand side and per grid of the current batch: slot index
    int32_t *d_rslot = nullptr, *d_gslot = nullptr;
    int32_t cap = 0;
    SpecSel sel64, sel32;
};

namespace {

// (exp(-jkR) - 1)/R for k = (1 - j)/delta, R >= 0; with a = R/delta the real part
// of the numerator is expm1(-a) cos a - 2 sin^2(a/2) (accurate for small a), and
// the value at R = 0 is the limit -(1 + j)/delta.
__device__ __forceinline__ double2 lossy_remainder(double R, double inv_delta) {
    if (!(R > 0.0)) return make_double2(-inv_delta, -inv_delta);
    const double a = R * inv_delta;
    double sn, cs;
    sincos(a, &sn, &cs);
    const double sh = sin(0.5 * a);
    const double re = expm1(-a) * cs - 2.0 * sh * sh;
    const double im = -exp(-a) * sn;
    return make_double2(re / R, im / R);
}

// Remainder block of the pair (T outer, S inner): 0.25 sum_p sum_q w_p w_q
// (r_p - v_k).(r'_q - v'_l) g(|r_p - r'_q|), written into blk[k][l] (only the
// entries with mask bit 3k + l set are accumulated, so the diagonal kernel can
// ask for one entry).
__device__ void remainder_block(const double *vT, const double *vS, const double *bary, const double *w,
                                double inv_delta, int mask, double2 *blk) {
    double rs[7][3];
    for (int q = 0; q < 7; ++q)
        for (int c = 0; c < 3; ++c)
            rs[q][c] = bary[3 * q] * vS[c] + bary[3 * q + 1] * vS[3 + c] + bary[3 * q + 2] * vS[6 + c];
    for (int i = 0; i < 9; ++i) blk[i] = make_double2(0.0, 0.0);
    for (int pq = 0; pq < 7; ++pq) {
        double r[3];
        for (int c = 0; c < 3; ++c) r[c] = bary[3 * pq] * vT[c] + bary[3 * pq + 1] * vT[3 + c] + bary[3 * pq + 2] * vT[6 + c];
        for (int q = 0; q < 7; ++q) {
            const double dx = r[0] - rs[q][0], dy = r[1] - rs[q][1], dz = r[2] - rs[q][2];
            const double2 g = lossy_remainder(sqrt(dx * dx + dy * dy + dz * dz), inv_delta);
            const double ww = w[pq] * w[q];
            for (int k = 0; k < 3; ++k) {
                const double o0 = r[0] - vT[3 * k], o1 = r[1] - vT[3 * k + 1], o2 = r[2] - vT[3 * k + 2];
                for (int l = 0; l < 3; ++l) {
                    if (!(mask >> (3 * k + l) & 1)) continue;
                    const double d = ww * (o0 * (rs[q][0] - vS[3 * l]) + o1 * (rs[q][1] - vS[3 * l + 1]) +
                                           o2 * (rs[q][2] - vS[3 * l + 2]));
                    blk[3 * k + l].x += d * g.x;
                    blk[3 * k + l].y += d * g.y;
                }
            }
        }
    }
    for (int i = 0; i < 9; ++i) blk[i] = make_double2(0.25 * blk[i].x, 0.25 * blk[i].y);
}

__device__ int64_t row_of(const int64_t *ptr, int64_t nrows, int64_t e) {
    int64_t lo = 0, hi = nrows;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) / 2;
        if (ptr[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

struct LossyNearArgs {
    const int64_t *ptr;
    const int32_t *col;
    int64_t nt;
    const double *verts;     // [nt][9]
    const double *r7b, *r7w;
    const double *Ldir;      // static direct blocks [n_near][9]
    const int32_t *start;    // [nt*Q][3]
    const double *lw;        // [nt*Q][3][O]
    const double *mom;       // [nt*Q][3][3]
    const double2 *Hpad;     // complex padded kernel [Mx][My][Mz]
    int Q, O, Mx, My, Mz;
    double inv_delta;
    double2 *Ld64;
    float2 *Ld32;
};

// One near pair per thread: L_d,k = L_direct + remainder - (I H_k B), the grid
// part being the double sum over the two stencils of every pair of sample
// points with the complex kernel table (grouped by node offset per axis).
__global__ void k_near_blocks_lossy(LossyNearArgs a, int64_t n_near) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n_near) return;
    const int64_t T = row_of(a.ptr, a.nt, e), S = a.col[e];
    double2 blk[9];
    remainder_block(a.verts + 9 * T, a.verts + 9 * S, a.r7b, a.r7w, a.inv_delta, 0x1ff, blk);
    const int Q = a.Q, O = a.O;
    double2 g[9];
    for (int i = 0; i < 9; ++i) g[i] = make_double2(0.0, 0.0);
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
            double Gr = 0.0, Gi = 0.0;
            for (int sx = 0; sx < 2 * O - 1; ++sx) {
                int dx = base[0] + sx;
                dx = ((dx % a.Mx) + a.Mx) % a.Mx;
                for (int sy = 0; sy < 2 * O - 1; ++sy) {
                    int dy = base[1] + sy;
                    dy = ((dy % a.My) + a.My) % a.My;
                    const double2 *row = a.Hpad + (int64_t(dx) * a.My + dy) * a.Mz;
                    const double cxy = cr[0][sx] * cr[1][sy];
                    double ar = 0.0, ai = 0.0;
                    for (int sz = 0; sz < 2 * O - 1; ++sz) {
                        int dz = base[2] + sz;
                        dz = ((dz % a.Mz) + a.Mz) % a.Mz;
                        ar += cr[2][sz] * row[dz].x;
                        ai += cr[2][sz] * row[dz].y;
                    }
                    Gr += cxy * ar;
                    Gi += cxy * ai;
                }
            }
            const double *fa = a.mom + 9 * pa, *fb = a.mom + 9 * pb;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    const double f = fa[3 * k] * fb[3 * l] + fa[3 * k + 1] * fb[3 * l + 1] + fa[3 * k + 2] * fb[3 * l + 2];
                    g[3 * k + l].x += f * Gr;
                    g[3 * k + l].y += f * Gi;
                }
        }
    }
    for (int i = 0; i < 9; ++i) {
        const double2 v = make_double2(a.Ldir[9 * e + i] + blk[i].x - g[i].x, blk[i].y - g[i].y);
        a.Ld64[9 * e + i] = v;
        a.Ld32[9 * e + i] = make_float2(float(v.x), float(v.y));
    }
}

// Lt_k[e][e] = sum over the branch's triangle pairs (T_a, T_b) of s_a s_b
// (L_direct + remainder)(T_a, T_b)[k_a][k_b], the static part read from the
// near list (every triangle pair of a branch is near), the remainder entry
// evaluated with T_a outer.
__global__ void k_branch_diag_lossy(const int64_t *ptr, const int32_t *col, const double *Ldir, const int32_t *br_tri,
                                    const int8_t *br_local, int64_t nb, const double *verts, const double *r7b,
                                    const double *r7w, double inv_delta, double2 *diag) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nb) return;
    const int32_t t[2] = {br_tri[2 * e], br_tri[2 * e + 1]};
    const int k[2] = {br_local[2 * e], br_local[2 * e + 1]};
    const double s[2] = {1.0, -1.0};
    double re = 0.0, im = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int64_t end = ptr[t[a] + 1];
            int64_t lo = ptr[t[a]], hi = end;
            while (lo < hi) {
                const int64_t mid = (lo + hi) / 2;
                if (col[mid] < t[b]) lo = mid + 1; else hi = mid;
            }
            if (!(lo < end && col[lo] == t[b])) continue;
            double2 blk[9];
            const int idx = 3 * k[a] + k[b];
            remainder_block(verts + 9 * t[a], verts + 9 * t[b], r7b, r7w, inv_delta, 1 << idx, blk);
            re += s[a] * s[b] * (Ldir[9 * lo + idx] + blk[idx].x);
            im += s[a] * s[b] * blk[idx].y;
        }
    diag[e] = make_double2(re, im);
}

int slot_alloc(pfft_plan *p, LossySlot &s) {
    if (s.H64) return SIE_OK;
    const int64_t nh = int64_t(p->Mx / 2 + 1) * (p->My / 2 + 1) * (p->Mz / 2 + 1);
    int rc;
    if ((rc = plan_alloc(p, (void **)&s.H64, nh * sizeof(double2)))) return rc;
    if ((rc = plan_alloc(p, (void **)&s.H32, nh * sizeof(float2)))) return rc;
    if ((rc = plan_alloc(p, (void **)&s.Ld64, size_t(p->n_near) * 9 * sizeof(double2)))) return rc;
    if ((rc = plan_alloc(p, (void **)&s.Ld32, size_t(p->n_near) * 9 * sizeof(float2)))) return rc;
    if ((rc = plan_alloc(p, (void **)&s.diagL, size_t(std::max<int64_t>(p->nb, 1)) * sizeof(double2)))) return rc;
    return SIE_OK;
}

// Builds slot i for angular frequency w on stream st (synchronises st).
int slot_build(pfft_plan *p, int i, double w, cudaStream_t st) {
    LossyCache &c = *p->lossy;
    LossySlot &s = c.slot[i];
    s.omega = -1.0;
    int rc = slot_alloc(p, s);
    if (rc) return rc;
    const double inv_delta = std::sqrt(w * kMu0 * p->sigma[0] / 2.0);
    const int64_t nM = int64_t(p->Mx) * p->My * p->Mz;
    double2 *Hc = nullptr;
    if ((rc = plan_alloc(p, (void **)&Hc, nM * sizeof(double2)))) return rc;
    auto done = [&](int r) {
        cudaStreamSynchronize(st);
        plan_free(p, Hc);
        return r;
    };
    if ((rc = lossy_fill_table(p, inv_delta, Hc, st))) return done(rc);
    if (p->n_near > 0) {
        LossyNearArgs a{p->d_near_ptr, p->d_near_col, p->nt, p->d_verts, p->d_r7b, p->d_r7w, p->d_Ldir64,
                        p->d_start, p->d_lw64, p->d_mom64, Hc, p->Q, p->O, p->Mx, p->My, p->Mz, inv_delta,
                        s.Ld64, s.Ld32};
        k_near_blocks_lossy<<<unsigned((p->n_near + 127) / 128), 128, 0, st>>>(a, p->n_near);
        p->launches++;
    }
    if (p->nb > 0) {
        k_branch_diag_lossy<<<unsigned((p->nb + 255) / 256), 256, 0, st>>>(
            p->d_near_ptr, p->d_near_col, p->d_Ldir64, p->d_br_tri, p->d_br_local, p->nb, p->d_verts, p->d_r7b,
            p->d_r7w, inv_delta, s.diagL);
        p->launches++;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return done(fail(SIE_ERR_CUDA, std::string("lossy near blocks: ") + cudaGetErrorString(e)));
    // the spectrum last: the transform may overwrite the table in place
    if ((rc = lossy_table_spectrum(p, Hc, s.H64, s.H32, st))) return done(rc);
    const void *ptrs[4] = {s.H64, s.H32, s.Ld64, s.Ld32};
    const void **tabs[4] = {c.d_htab64, c.d_htab32, c.d_ltab64, c.d_ltab32};
    for (int t = 0; t < 4; ++t)
        if ((e = cudaMemcpyAsync(tabs[t] + i, &ptrs[t], sizeof(void *), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return done(fail(SIE_ERR_CUDA, std::string("lossy slot tables: ") + cudaGetErrorString(e)));
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return done(fail(SIE_ERR_CUDA, std::string("lossy slot: ") + cudaGetErrorString(e)));
    s.omega = w;
    return done(SIE_OK);
}

int cache_init(pfft_plan *p) {
    if (p->lossy) return SIE_OK;
    p->lossy = new (std::nothrow) LossyCache;
    if (!p->lossy) return fail(SIE_ERR_OOM, "lossy kernel: out of host memory");
    LossyCache &c = *p->lossy;
    const void ***tabs[4] = {&c.d_htab64, &c.d_htab32, &c.d_ltab64, &c.d_ltab32};
    for (auto t : tabs) {
        int rc = plan_alloc(p, (void **)t, kLossyMaxSlots * sizeof(void *));
        if (rc) return rc;
        SIE_CUDA(cudaMemset(*t, 0, kLossyMaxSlots * sizeof(void *)));
    }
    return SIE_OK;
}

// Slot of w, building it (in an empty slot, or in the least recently used one
// that the current batch does not use) when it is not cached.
int slot_of(pfft_plan *p, double w, const std::vector<char> &in_use, cudaStream_t st, int &out) {
    LossyCache &c = *p->lossy;
    for (int i = 0; i < kLossyMaxSlots; ++i)
        if (c.slot[i].omega == w) { out = i; return SIE_OK; }
    int pick = -1;
    for (int i = 0; i < kLossyMaxSlots && pick < 0; ++i)   // an empty slot first
        if (c.slot[i].omega < 0.0 && !in_use[i]) pick = i;
    if (pick < 0)                                           // else the least recently used one not in use
        for (int i = 0; i < kLossyMaxSlots; ++i)
            if (!in_use[i] && (pick < 0 || c.slot[i].last_use < c.slot[pick].last_use)) pick = i;
    if (pick < 0)
        return fail(SIE_ERR_ARG, "lossy kernel: more than " + std::to_string(kLossyMaxSlots) +
                                     " distinct frequencies in one call");
    int rc = slot_build(p, pick, w, st);
    if (rc) return rc;
    out = pick;
    return SIE_OK;
}

}  // namespace

int lossy_prepare(pfft_plan *p, const double *omega, int32_t R, cudaStream_t st) {
    int rc = cache_init(p);
    if (rc) return rc;
    LossyCache &c = *p->lossy;
    std::vector<char> in_use(kLossyMaxSlots, 0);
    std::vector<int32_t> rslot(R);
    for (int32_t r = 0; r < R; ++r) {
        const double w = omega[r];
        if (!(w > 0.0) || !std::isfinite(w))
            return fail(SIE_ERR_ARG, "pfft_matvec: the lossy kernel needs omega finite and > 0");
        int i = -1;
        if (r > 0 && omega[r - 1] == w) i = rslot[r - 1];
        else if ((rc = slot_of(p, w, in_use, st, i))) return rc;
        rslot[r] = i;
        in_use[i] = 1;
        c.slot[i].last_use = ++c.tick;
    }
    if (c.cap < R) {
        if (c.d_rslot) plan_free(p, c.d_rslot);
        if (c.d_gslot) plan_free(p, c.d_gslot);
        c.d_rslot = c.d_gslot = nullptr;
        c.cap = 0;
        if ((rc = plan_alloc(p, (void **)&c.d_rslot, size_t(R) * sizeof(int32_t)))) return rc;
        if ((rc = plan_alloc(p, (void **)&c.d_gslot, size_t(3) * R * sizeof(int32_t)))) return rc;
        c.cap = R;
    }
    // grids are [3][R]: grid c R + r belongs to right-hand side r
    std::vector<int32_t> gslot(size_t(3) * R);
    for (int d = 0; d < 3; ++d) std::copy(rslot.begin(), rslot.end(), gslot.begin() + size_t(d) * R);
    SIE_CUDA(cudaMemcpyAsync(c.d_rslot, rslot.data(), size_t(R) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    SIE_CUDA(cudaMemcpyAsync(c.d_gslot, gslot.data(), gslot.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    c.sel64 = SpecSel{c.d_htab64, c.d_gslot};
    c.sel32 = SpecSel{c.d_htab32, c.d_gslot};
    return SIE_OK;
}

const SpecSel *lossy_sel(const pfft_plan *p, int prec) {
    return prec == SIE_PREC_FP64 ? &p->lossy->sel64 : &p->lossy->sel32;
}
const void *const *lossy_ltab(const pfft_plan *p, int prec) {
    return prec == SIE_PREC_FP64 ? p->lossy->d_ltab64 : p->lossy->d_ltab32;
}
const int32_t *lossy_rslot(const pfft_plan *p) { return p->lossy->d_rslot; }

int lossy_diag(pfft_plan *p, const double *omega, int32_t ns, double2 *out, cudaStream_t st) {
    int rc = cache_init(p);
    if (rc) return rc;
    LossyCache &c = *p->lossy;
    std::vector<char> in_use(kLossyMaxSlots, 0);
    for (int32_t f = 0; f < ns; ++f) {
        int i = -1;
        if ((rc = slot_of(p, omega[f], in_use, st, i))) return rc;
        in_use[i] = 1;
        c.slot[i].last_use = ++c.tick;
        SIE_CUDA(cudaMemcpyAsync(out + size_t(f) * p->nb, c.slot[i].diagL, size_t(p->nb) * sizeof(double2),
                                 cudaMemcpyDeviceToDevice, st));
    }
    return SIE_OK;
}

void plan_free_lossy(pfft_plan *p) {
    delete p->lossy;   // its device buffers are plan allocations, freed with the plan
    p->lossy = nullptr;
}

}  // namespace sie
