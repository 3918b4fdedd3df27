// Tables of the double-float product (SIE_PREC_DF), rounded once from the FP64
// tables of the plan: the projection / interpolation and near-field block
// records (Eq. Projection, Eq. interpolation, Eq. Lb), the four-step twiddles
// of the three axes and the folded kernel spectrum (Eq. FFTCal).  Each FP64
// value v becomes the pair hi = fl32(v), lo = fl32(v - hi), which carries v to
// about 2^-48 relative; the product's kernels then run on the FP32 pipes.
#include <algorithm>

#include "sie_plan.h"

using namespace sie;

namespace {

__device__ __forceinline__ df to_df(double v) {
    const float hi = __double2float_rn(v);
    return df(hi, __double2float_rn(v - double(hi)));
}

__global__ void k_rec_to_df(const Rec<double> *__restrict__ in, Rec<df> *__restrict__ out, int64_t n) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Rec<df> r;
#pragma unroll
    for (int k = 0; k < 9; ++k) r.b[k] = to_df(in[i].b[k]);
    r.col = int32_t(in[i].col);
    r.pad = 0;
    out[i] = r;
}

__global__ void k_c_to_df(const double2 *__restrict__ in, cdf *__restrict__ out, int64_t n) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = in[i];
    cdf o;
    o.x = to_df(v.x);
    o.y = to_df(v.y);
    out[i] = o;
}

__global__ void k_r_to_df(const double *__restrict__ in, df *__restrict__ out, int64_t n) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = to_df(in[i]);
}

unsigned nblk(int64_t n) { return unsigned((n + 255) / 256); }

}  // namespace

namespace sie {

int df_prepare(pfft_plan *p, cudaStream_t st) {
    if (p->df_ready) return SIE_OK;
    if (!p->d_pn_rec64 || !p->d_pt_rec64 || !p->d_near_rec64 || !p->d_Hp64)
        return fail(SIE_ERR_ARG, "double-float product: the plan has no FP64 tables to round");
    int rc;
    auto recs = [&](const Rec<double> *src, Rec<df> **dst, int64_t n) -> int {
        if ((rc = plan_alloc(p, (void **)dst, size_t(std::max<int64_t>(n, 1)) * sizeof(Rec<df>)))) return rc;
        if (n > 0) {
            k_rec_to_df<<<nblk(n), 256, 0, st>>>(src, *dst, n);
            SIE_LAUNCH_CHECK(p);
        }
        return SIE_OK;
    };
    if ((rc = recs(p->d_pn_rec64, &p->d_pn_recdf, p->n_pair))) return rc;
    if ((rc = recs(p->d_pt_rec64, &p->d_pt_recdf, p->n_pair))) return rc;
    if ((rc = recs(p->d_near_rec64, &p->d_near_recdf, p->n_near))) return rc;
    const int M[3] = {p->Mx, p->My, p->Mz};
    for (int a = 0; a < 3; ++a) {
        for (int inv = 0; inv < 2; ++inv) {
            const double2 *src = inv ? p->d_ti64[a] : p->d_tf64[a];
            cdf **dst = inv ? &p->d_tidf[a] : &p->d_tfdf[a];
            if ((rc = plan_alloc(p, (void **)dst, size_t(M[a]) * sizeof(cdf)))) return rc;
            k_c_to_df<<<nblk(M[a]), 256, 0, st>>>(src, *dst, M[a]);
            SIE_LAUNCH_CHECK(p);
        }
    }
    const int64_t nh = int64_t(p->Mx / 2 + 1) * (p->My / 2 + 1) * (p->Mz / 2 + 1);
    if ((rc = plan_alloc(p, (void **)&p->d_Hpdf, size_t(nh) * sizeof(df)))) return rc;
    k_r_to_df<<<nblk(nh), 256, 0, st>>>(p->d_Hp64, p->d_Hpdf, nh);
    SIE_LAUNCH_CHECK(p);
    p->df_ready = true;
    return SIE_OK;
}

}  // namespace sie
