// pfft_autotune: the pFFT grid of a geometry picked by measurement.
//
// The grid spacing trades the far field's FFT cost (grows with the node count)
// against the near field's cost (the pre-corrected near list grows with the
// spacing, since pairs within near_factor spacings or with overlapping stencils
// are near) and against accuracy (Sec. IV-B: the grid product approximates
// the far interactions).  Candidates are the base grid, half and double it on
// every axis, and the base with one axis doubled; each is built, its mixed
// matvec timed with CUDA events on the caller's stream at the caller's
// right-hand-side count, and its FP64 product compared with that of the finest
// candidate built with a near radius half again as large (the reference).  The
// fastest candidate within `tol` of the reference wins.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sie_plan.h"

using namespace sie;

namespace {

// splitmix64: deterministic test vectors without the host's RNG state
uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
double uniform(uint64_t i) { return double(mix64(i) >> 11) * (1.0 / 9007199254740992.0) - 0.5; }

bool grid_ok(const int g[3], int order) {
    for (int d = 0; d < 3; ++d)
        if (g[d] < std::max(4, order) || g[d] > 256 || (g[d] & (g[d] - 1))) return false;
    return true;
}

struct TuneBuf {
    void *p = nullptr;
    ~TuneBuf() { if (p) cudaFree(p); }
};

}  // namespace

extern "C" int pfft_autotune(const sie_mesh *m, const sie_loops *l, const pfft_params *base, int32_t nrhs,
                             double omega, double tol, void *cuda_stream, pfft_params *best,
                             sie_tune_report *rep) {
    if (!m || !l || !base || !best || nrhs < 1 || !(omega > 0.0) || !(tol > 0.0))
        return fail(SIE_ERR_ARG, "pfft_autotune: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // candidate grids
    std::vector<std::array<int, 3>> cand;
    auto add = [&](int a, int b, int c) {
        const int g[3] = {a, b, c};
        if (!grid_ok(g, base->order)) return;
        for (auto &x : cand) if (x[0] == a && x[1] == b && x[2] == c) return;
        cand.push_back({a, b, c});
    };
    const int *g0 = base->grid;
    add(g0[0], g0[1], g0[2]);
    add(g0[0] / 2, g0[1] / 2, g0[2] / 2);
    add(2 * g0[0], 2 * g0[1], 2 * g0[2]);
    add(2 * g0[0], g0[1], g0[2]);
    add(g0[0], 2 * g0[1], g0[2]);
    add(g0[0], g0[1], 2 * g0[2]);
    if (cand.empty()) return fail(SIE_ERR_ARG, "pfft_autotune: the base grid is out of range");
    if (int(cand.size()) > SIE_TUNE_MAX) cand.resize(SIE_TUNE_MAX);
    // reference: the finest candidate, near radius x 1.5
    size_t fine = 0;
    for (size_t i = 1; i < cand.size(); ++i)
        if (int64_t(cand[i][0]) * cand[i][1] * cand[i][2] > int64_t(cand[fine][0]) * cand[fine][1] * cand[fine][2])
            fine = i;
    const int64_t nl = l->nl;
    const size_t vbytes = size_t(nrhs) * nl * sizeof(double2);
    std::vector<double2> hx(size_t(nrhs) * nl);
    for (size_t i = 0; i < hx.size(); ++i) hx[i] = make_double2(uniform(2 * i), uniform(2 * i + 1));
    std::vector<double> om(nrhs, omega);
    TuneBuf x, y, yref;
    SIE_CUDA(cudaMalloc(&x.p, vbytes));
    SIE_CUDA(cudaMalloc(&y.p, vbytes));
    SIE_CUDA(cudaMalloc(&yref.p, vbytes));
    SIE_CUDA(cudaMemcpy(x.p, hx.data(), vbytes, cudaMemcpyHostToDevice));
    int rc;
    {
        pfft_params pr = *base;
        for (int d = 0; d < 3; ++d) pr.grid[d] = cand[fine][d];
        pr.near_factor = base->near_factor * 1.5;
        pfft_plan *P = nullptr;
        if ((rc = pfft_plan_create(m, l, &pr, cuda_stream, &P))) return rc;
        rc = pfft_matvec(P, x.p, yref.p, nrhs, om.data(), SIE_SPACE_LOOP, SIE_PREC_FP64, cuda_stream);
        pfft_plan_destroy(P);
        if (rc) return rc;
    }
    std::vector<double2> href(hx.size()), hy(hx.size());
    SIE_CUDA(cudaMemcpy(href.data(), yref.p, vbytes, cudaMemcpyDeviceToHost));
    sie_tune_report r{};
    r.n_tried = int32_t(cand.size());
    r.best = -1;
    cudaEvent_t e0, e1;
    SIE_CUDA(cudaEventCreate(&e0));
    SIE_CUDA(cudaEventCreate(&e1));
    auto done = [&](int code) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return code;
    };
    for (size_t c = 0; c < cand.size(); ++c) {
        pfft_params pr = *base;
        for (int d = 0; d < 3; ++d) pr.grid[d] = r.grid[c][d] = cand[c][d];
        pfft_plan *P = nullptr;
        if ((rc = pfft_plan_create(m, l, &pr, cuda_stream, &P))) return done(rc);
        // accuracy: FP64 product against the reference
        rc = pfft_matvec(P, x.p, y.p, nrhs, om.data(), SIE_SPACE_LOOP, SIE_PREC_FP64, cuda_stream);
        if (!rc && cudaMemcpy(hy.data(), y.p, vbytes, cudaMemcpyDeviceToHost) != cudaSuccess) rc = SIE_ERR_CUDA;
        double err = 0.0;
        for (int32_t k = 0; k < nrhs && !rc; ++k) {
            double num = 0.0, den = 0.0;
            for (int64_t i = 0; i < nl; ++i) {
                const double2 a = hy[k * nl + i], b = href[k * nl + i];
                num += (a.x - b.x) * (a.x - b.x) + (a.y - b.y) * (a.y - b.y);
                den += b.x * b.x + b.y * b.y;
            }
            err = std::max(err, std::sqrt(num / std::max(den, 1e-300)));
        }
        // time: mixed matvecs on the caller's stream after two warm-ups
        constexpr int kReps = 5;
        float ms = 0.f;
        for (int w = 0; w < 2 && !rc; ++w)
            rc = pfft_matvec(P, x.p, y.p, nrhs, om.data(), SIE_SPACE_LOOP, SIE_PREC_MIXED, cuda_stream);
        if (!rc) {
            cudaEventRecord(e0, st);
            for (int k = 0; k < kReps && !rc; ++k)
                rc = pfft_matvec(P, x.p, y.p, nrhs, om.data(), SIE_SPACE_LOOP, SIE_PREC_MIXED, cuda_stream);
            cudaEventRecord(e1, st);
            if (!rc && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        }
        pfft_plan_destroy(P);
        if (rc) return done(rc);
        r.ms[c] = double(ms) / kReps;
        r.err[c] = err;
        if (err <= tol && (r.best < 0 || r.ms[c] < r.ms[r.best])) r.best = int32_t(c);
    }
    *best = *base;
    if (r.best >= 0) {
        for (int d = 0; d < 3; ++d) best->grid[d] = r.grid[r.best][d];
    } else {   // nothing within tol: the reference grid and radius
        for (int d = 0; d < 3; ++d) best->grid[d] = cand[fine][d];
        best->near_factor = base->near_factor * 1.5;
    }
    if (rep) *rep = r;
    return done(SIE_OK);
}

extern "C" int pfft_plan_set_kernel_tuning(pfft_plan *p, const sie_kernel_tuning *t) {
    if (!p) return fail(SIE_ERR_ARG, "pfft_plan_set_kernel_tuning: NULL plan");
    sie_kernel_tuning k{};
    if (t) k = *t;
    if (k.near < 0 || k.near > 2 || (k.far_slab != 0 && k.far_slab != 64 && k.far_slab != 128) ||
        (k.proj_slab != 0 && k.proj_slab != 32 && k.proj_slab != 64 && k.proj_slab != 128) || k.plane_gpc < 0 ||
        k.plane_gpc > 8)
        return fail(SIE_ERR_ARG, "pfft_plan_set_kernel_tuning: value out of range");
    p->kt = k;
    return SIE_OK;
}

extern "C" int pfft_plan_get_kernel_tuning(const pfft_plan *p, sie_kernel_tuning *t) {
    if (!p || !t) return fail(SIE_ERR_ARG, "pfft_plan_get_kernel_tuning: NULL argument");
    *t = p->kt;
    return SIE_OK;
}

extern "C" int pfft_autotune_kernels(pfft_plan *p, int32_t nrhs, double omega, void *cuda_stream,
                                     sie_kernel_tuning *best, sie_kernel_tune_report *rep) {
    if (!p || nrhs < 1 || !(omega > 0.0) || !std::isfinite(omega))
        return fail(SIE_ERR_ARG, "pfft_autotune_kernels: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the near paths that apply at this count: automatic, and the other one when the
    // count is even (the tensor-core path needs an even count)
    std::vector<int32_t> nears{0};
    if (nrhs % 2 == 0) nears.push_back(nrhs >= 96 ? 2 : 1);
    std::vector<sie_kernel_tuning> cand;
    for (int32_t nr : nears)
        for (int32_t fs : {64, 128})
            for (int32_t ps : {32, 64, 128})
                for (int32_t g : {0, 4}) cand.push_back(sie_kernel_tuning{nr, fs, ps, g});
    if (int(cand.size()) > SIE_KTUNE_MAX) cand.resize(SIE_KTUNE_MAX);
    const int64_t nl = p->nl;
    const size_t vbytes = size_t(nrhs) * nl * sizeof(double2);
    std::vector<double2> hx(size_t(nrhs) * nl);
    for (size_t i = 0; i < hx.size(); ++i) hx[i] = make_double2(uniform(2 * i + 7), uniform(2 * i + 8));
    std::vector<double> om(nrhs, omega);
    TuneBuf x, y;
    SIE_CUDA(cudaMalloc(&x.p, vbytes));
    SIE_CUDA(cudaMalloc(&y.p, vbytes));
    SIE_CUDA(cudaMemcpy(x.p, hx.data(), vbytes, cudaMemcpyHostToDevice));
    const sie_kernel_tuning keep = p->kt;
    sie_kernel_tune_report r{};
    r.n_tried = int32_t(cand.size());
    r.best = -1;
    cudaEvent_t e0, e1;
    SIE_CUDA(cudaEventCreate(&e0));
    SIE_CUDA(cudaEventCreate(&e1));
    auto done = [&](int code) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (code) p->kt = keep;
        return code;
    };
    for (size_t c = 0; c < cand.size(); ++c) {
        p->kt = cand[c];
        r.cand[c] = cand[c];
        int rc = SIE_OK;
        for (int w = 0; w < 2 && !rc; ++w)
            rc = pfft_matvec(p, x.p, y.p, nrhs, om.data(), SIE_SPACE_LOOP, SIE_PREC_MIXED, cuda_stream);
        float ms = 0.f;
        if (!rc) {
            constexpr int kReps = 5;
            cudaEventRecord(e0, st);
            for (int k = 0; k < kReps && !rc; ++k)
                rc = pfft_matvec(p, x.p, y.p, nrhs, om.data(), SIE_SPACE_LOOP, SIE_PREC_MIXED, cuda_stream);
            cudaEventRecord(e1, st);
            if (!rc && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            ms /= kReps;
        }
        if (rc) return done(rc);
        r.ms[c] = ms;
        if (r.best < 0 || r.ms[c] < r.ms[r.best]) r.best = int32_t(c);
    }
    p->kt = cand[r.best];
    if (best) *best = p->kt;
    if (rep) *rep = r;
    return done(SIE_OK);
}
