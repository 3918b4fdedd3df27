// Instantiations and launcher of the paired FP32 plane convolution
// (sie_plane.cuh) for every padded plane My x Mz the plan accepts (powers of
// two, 8..256, My Mz <= 8192; at most 99 KB of shared memory, two CTAs per SM).
#include <algorithm>

#include "sie_plan.h"
#include "sie_plane.cuh"

namespace sie {
namespace {

template <int MY, int MZ>
int launch_plane(pfft_plan *p, float2 *spec, int32_t ngrids, int lgMx, cudaStream_t s) {
    using G = plane::Geo<MY, MZ>;
    auto kern = plane::k_plane_conv<MY, MZ>;
    if (int rc = set_smem((const void *)kern, G::kSmem)) return rc;
    int nsm = 0;
    SIE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
    // grids per CTA: up to 8 (the staged spectrum and twiddles serve each of
    // them) while keeping about four waves of two CTAs per SM
    const int64_t planes = int64_t(ngrids) * p->Mx;
    const int cap = p->kt.plane_gpc > 0 ? p->kt.plane_gpc : 8;
    const int gpc = int(std::max<int64_t>(1, std::min<int64_t>(cap, planes / (8 * int64_t(nsm)))));
    const int64_t ctas = int64_t(p->Mx) * ((ngrids + gpc - 1) / gpc);
    kern<<<unsigned(ctas), plane::kThreads, G::kSmem, s>>>(spec, ngrids, gpc, lgMx, p->d_Hp32, p->d_tf32[1],
                                                           p->d_ti32[1], p->d_tf32[2], p->d_ti32[2]);
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

template <int MY>
int dispatch_mz(pfft_plan *p, float2 *spec, int32_t ngrids, int lgMx, cudaStream_t s, bool &done) {
    done = true;
    switch (p->Mz) {
        case 8: return launch_plane<MY, 8>(p, spec, ngrids, lgMx, s);
        case 16: return launch_plane<MY, 16>(p, spec, ngrids, lgMx, s);
        case 32: return launch_plane<MY, 32>(p, spec, ngrids, lgMx, s);
        case 64: return launch_plane<MY, 64>(p, spec, ngrids, lgMx, s);
        case 128:
            if constexpr (MY <= 64) return launch_plane<MY, 128>(p, spec, ngrids, lgMx, s);
            break;
        case 256:
            if constexpr (MY <= 32) return launch_plane<MY, 256>(p, spec, ngrids, lgMx, s);
            break;
        default: break;
    }
    done = false;
    return SIE_OK;
}

}  // namespace

bool plane_conv_supported(const pfft_plan *p) {
    auto pow2 = [](int v) { return v >= 8 && v <= 256 && (v & (v - 1)) == 0; };
    return p->d_Hp32 && pow2(p->My) && pow2(p->Mz) && int64_t(p->My) * p->Mz <= 8192;
}

int plane_conv_f32(pfft_plan *p, float2 *spec, int32_t ngrids, cudaStream_t s, bool &done) {
    done = false;
    if (!plane_conv_supported(p)) return SIE_OK;
    int lgMx = 0;
    while ((1 << lgMx) < p->Mx) ++lgMx;
    switch (p->My) {
        case 8: return dispatch_mz<8>(p, spec, ngrids, lgMx, s, done);
        case 16: return dispatch_mz<16>(p, spec, ngrids, lgMx, s, done);
        case 32: return dispatch_mz<32>(p, spec, ngrids, lgMx, s, done);
        case 64: return dispatch_mz<64>(p, spec, ngrids, lgMx, s, done);
        case 128: return dispatch_mz<128>(p, spec, ngrids, lgMx, s, done);
        case 256: return dispatch_mz<256>(p, spec, ngrids, lgMx, s, done);
        default: return SIE_OK;
    }
}

}  // namespace sie
