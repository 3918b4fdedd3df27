// Preconditioner and solver of Sec. IV-A (arXiv 2210.04891).
//
// Eq. (Precond): P = A Z_b^N A^T, Z_b^N = diag(Z_b) (port links carry no
// impedance).  P^-1 y is applied exactly through the nodal form of the same
// circuit: with D = diag(Z_b) every branch e is an impedance D_e, each link
// carries the loop's EMF y_l, each port is an ideal source of EMF y_p between
// its sink and source nodes.  Node potentials phi solve the weighted graph
// Laplacian  sum_e (1/D_e)(phi_tail - phi_head + emf_e) = 0  per node (one
// grounded node per conductor, source nodes fixed by their port EMF); the link
// currents (1/D_e)(phi_tail - phi_head + emf_e) and the port currents are then
// z = P^-1 y.  This equals the loop-space solve because the fundamental loops
// span exactly the currents that satisfy Kirchhoff's current law.  The
// Laplacian is far sparser than P (a triangle has three neighbours) and does
// not depend on the spanning tree.  Each conductor's Laplacian is ordered by
// reverse Cuthill-McKee and factorised as a band LDL^T without pivoting (its
// Hermitian part, the Laplacian of Re(1/D_e) > 0, is positive definite).
//
// Eq. (LoopWithP): restarted GMRES on P^-1 Z_l I_l = P^-1 V_l for all
// (frequency, port) right-hand sides at once; Arnoldi by classical
// Gram-Schmidt applied twice, in FP64 on the device; Givens rotations and the
// small least-squares solve on the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <deque>
#include <map>
#include <numeric>
#include <type_traits>
#include <vector>

#include "sie_plan.h"

using namespace sie;

namespace sie {
int matvec_async(pfft_plan *p, const void *x, void *y, int32_t nrhs, const double *omega, int space, int prec,
                 cudaStream_t st);

// Bands from 32 to kWideMax - 1 wide use the CTA-wide sweeps (one thread per window row).
constexpr int32_t kWideMax = 1024;

struct PrecondState {
    // symbolic (host-built once)
    int64_t nunk = 0;                 // unknowns (permuted, concatenated by block)
    int32_t W = 0;                    // band width (max over blocks)
    std::vector<int64_t> blk_off;     // [nblk + 1] unknown offset of each block
    int32_t *d_blk_off32 = nullptr;
    int64_t *d_blk_off = nullptr;
    int32_t *d_unk_of_node = nullptr;  // [nn] permuted unknown index, -1 fixed
    int32_t *d_off_ptr = nullptr, *d_off_port = nullptr;  // node -> (port, sign) potential offsets
    int8_t *d_off_sign = nullptr;
    int32_t *d_row_ptr = nullptr, *d_row_br = nullptr;    // unknown row -> incident branches
    int8_t *d_row_sg = nullptr;                            // +1 tail in row's group, -1 head
    int32_t *d_row_oth = nullptr;                          // other end's unknown (-1 fixed / same)
    int32_t *d_src_ptr = nullptr, *d_src_br = nullptr;     // port -> branches at its source node
    int8_t *d_src_sg = nullptr;
    int32_t *d_port_loop = nullptr;
    // numeric
    int32_t nslots = 0;
    std::vector<double> slot_omega;
    double2 *d_band = nullptr;        // [nslots][nunk][W + 1], band[i][d] = K[i][i-d]
    double2 *d_bandc = nullptr;       // same, column-major copy bandc[i][d] = L[i+d][i]
    // sweep tiles (band width <= 31, see k_pc_tiles) in FP64 and FP32, reciprocal pivots
    std::vector<int64_t> tile_off;    // [nblk + 1] first chunk of each block
    int64_t *d_tile_off = nullptr;
    int64_t nchunks = 0;
    double2 *d_tile64 = nullptr, *d_dinv64 = nullptr;
    float2 *d_tile32 = nullptr, *d_dinv32 = nullptr;
    cdf *d_tiledf = nullptr, *d_dinvdf = nullptr;   // double-float sweeps (SIE_PREC_DF)
    float2 *d_u32 = nullptr;          // FP32 sweep buffer [R][nunk]
    // bands wider than a warp (31 < W < 1024): FP32 roundings of band and bandc (mixed form)
    float2 *d_band32 = nullptr, *d_bandc32 = nullptr;
    double2 *d_a = nullptr;           // [nslots][nb] 1/D_e
    float2 *d_a32 = nullptr;          // its FP32 rounding (mixed form)
    cdf *d_adf = nullptr;             // its double-float rounding (narrow bands)
    double2 *d_kappa = nullptr, *d_u = nullptr, *d_ibr = nullptr;   // scratch [R][...]
    int32_t cap_rhs = 0;
    int32_t *d_slot = nullptr;        // [R] factor slot per right-hand side
    int *d_status = nullptr;
    // nested-dissection route (bands too wide, or asked for): the multifrontal factors of
    // every slot [nslots][sumL] in FP64 and FP32, and the solves' update vectors [R][sumU]
    NdState *nd = nullptr;
    double2 *d_ndL64 = nullptr;
    float2 *d_ndL32 = nullptr;
    double2 *d_uv = nullptr;
    int32_t *d_grp = nullptr;         // [ngrp][group size] right-hand sides sharing a slot (-1 pads)
    int32_t ngrp = 0, cap_grp = 0;
    std::vector<void *> allocs;
};

// The plan's memory pool (created on first use).  Stream-ordered allocations from
// it do not synchronise the device, and with an unbounded release threshold the
// memory a solve frees stays mapped for the next one.
cudaError_t plan_pool(pfft_plan *p, cudaMemPool_t *out) {
    if (!p->pool) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = p->device;
        cudaError_t e = cudaMemPoolCreate(&p->pool, &props);
        if (e != cudaSuccess) { p->pool = nullptr; return e; }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(p->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    *out = p->pool;
    return cudaSuccess;
}

template <typename Ptr>
cudaError_t pool_alloc(pfft_plan *p, Ptr **ptr, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool;
    cudaError_t e = plan_pool(p, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync((void **)ptr, bytes, pool, st);
}

// DC (omega = 0) has a solution only when every conductor has a slab surface
// model: the classic Z_s and c_L both vanish there.
bool dc_defined(const pfft_plan *p) {
    for (double t : p->t_eff)
        if (!(t > 0.0)) return false;
    return !p->t_eff.empty();
}

void plan_free_precond(pfft_plan *p) {
    if (!p || !p->pc) return;
    for (void *a : p->pc->allocs) cudaFree(a);
    for (void *a : {(void *)p->pc->d_tile64, (void *)p->pc->d_dinv64, (void *)p->pc->d_tile32,
                    (void *)p->pc->d_dinv32, (void *)p->pc->d_u32, (void *)p->pc->d_a32,
                    (void *)p->pc->d_band32, (void *)p->pc->d_bandc32, (void *)p->pc->d_tiledf,
                    (void *)p->pc->d_dinvdf, (void *)p->pc->d_adf})
        if (a) cudaFree(a);
    for (void *a : {(void *)p->pc->d_band, (void *)p->pc->d_bandc, (void *)p->pc->d_a, (void *)p->pc->d_kappa, (void *)p->pc->d_u,
                    (void *)p->pc->d_ibr, (void *)p->pc->d_slot, (void *)p->pc->d_ndL64, (void *)p->pc->d_ndL32,
                    (void *)p->pc->d_uv, (void *)p->pc->d_grp})
        if (a) cudaFree(a);
    nd_free(p->pc->nd);
    delete p->pc;
    p->pc = nullptr;
}
}  // namespace sie

namespace {

constexpr double kMu0 = 4e-7 * M_PI;

template <typename T>
int pc_upload(PrecondState *s, T **dst, const std::vector<T> &v) {
    size_t b = std::max<size_t>(v.size() * sizeof(T), 16);
    SIE_CUDA(cudaMalloc((void **)dst, b));
    s->allocs.push_back(*dst);
    if (!v.empty()) SIE_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SIE_OK;
}

// Symbolic set-up: grounds, port offsets, unknown numbering (RCM per block),
// row -> branch lists.
int build_symbolic(pfft_plan *p) {
    const sie_loops *L = p->loops;
    const int64_t nn = L->n_nodes, nb = L->nb, np = L->np;
    auto *s = new (std::nothrow) PrecondState;
    if (!s) return fail(SIE_ERR_OOM, "preconditioner: out of host memory");
    p->pc = s;
    // port groups: nodes linked by port sources (union-find), offsets by BFS
    std::vector<std::vector<std::pair<int32_t, int32_t>>> padj(nn);   // (other node, +-(port+1))
    for (int64_t q = 0; q < np; ++q) {
        int32_t snk = L->port_sink[q], src = L->port_src[q];
        padj[snk].emplace_back(src, int32_t(q + 1));     // phi_src = phi_snk + y_q
        padj[src].emplace_back(snk, -int32_t(q + 1));
    }
    for (int64_t q = 0; q < np; ++q)
        for (int64_t r = 0; r < np; ++r)
            if (q != r && (L->port_src[q] == L->port_src[r] || L->port_src[q] == L->port_sink[r]))
                return fail(SIE_ERR_BAD_PORT, "preconditioner: a port's source contact is shared with another port");
    std::vector<int32_t> group(nn, -1);
    std::vector<std::vector<std::pair<int32_t, int8_t>>> off(nn);
    std::vector<int32_t> ground_of_comp(L->n_comp, -1);
    for (int64_t q = 0; q < np; ++q)
        if (ground_of_comp[L->comp[L->port_sink[q]]] < 0) ground_of_comp[L->comp[L->port_sink[q]]] = L->port_sink[q];
    for (int64_t v = 0; v < nn; ++v)
        if (ground_of_comp[L->comp[v]] < 0) ground_of_comp[L->comp[v]] = int32_t(v);
    std::vector<char> fixed(nn, 0);
    int32_t ngroups = 0;
    for (int64_t v0 = 0; v0 < nn; ++v0) {
        if (group[v0] >= 0 || padj[v0].empty()) continue;
        // BFS over port edges from v0
        std::vector<int32_t> members{int32_t(v0)};
        group[v0] = ngroups;
        for (size_t k = 0; k < members.size(); ++k) {
            int32_t u = members[k];
            for (auto [w, sp] : padj[u]) {
                if (group[w] >= 0) {
                    if (group[w] != ngroups) return fail(SIE_ERR_BAD_PORT, "preconditioner: inconsistent port groups");
                    continue;
                }
                group[w] = ngroups;
                off[w] = off[u];
                off[w].emplace_back(std::abs(sp) - 1, int8_t(sp > 0 ? 1 : -1));
                members.push_back(w);
            }
        }
        if (members.size() > size_t(np) + 1)
            return fail(SIE_ERR_BAD_PORT, "preconditioner: ports form a closed loop of sources");
        // rebase offsets on the group's ground if it holds one
        int32_t g = ground_of_comp[L->comp[v0]];
        if (group[g] == ngroups) {
            auto base = off[g];
            for (int32_t m : members) {
                for (auto [q, sg] : base) off[m].emplace_back(q, int8_t(-sg));
                fixed[m] = 1;
            }
        }
        ++ngroups;
    }
    for (int64_t c = 0; c < L->n_comp; ++c) fixed[ground_of_comp[c]] = 1;
    // unknowns: one per free group (its members share it), one per other free node
    std::vector<int32_t> unk_raw(nn, -1);
    std::vector<int32_t> group_unk(ngroups, -1);
    int64_t nunk = 0;
    for (int64_t v = 0; v < nn; ++v) {
        if (fixed[v]) continue;
        if (group[v] >= 0) {
            if (group_unk[group[v]] < 0) group_unk[group[v]] = int32_t(nunk++);
            unk_raw[v] = group_unk[group[v]];
        } else {
            unk_raw[v] = int32_t(nunk++);
        }
    }
    s->nunk = nunk;
    // unknown adjacency
    std::vector<std::vector<int32_t>> uadj(nunk);
    for (int64_t e = 0; e < nb; ++e) {
        int32_t a = unk_raw[L->tail[e]], b = unk_raw[L->head[e]];
        if (a >= 0 && b >= 0 && a != b) { uadj[a].push_back(b); uadj[b].push_back(a); }
    }
    for (auto &v : uadj) { std::sort(v.begin(), v.end()); v.erase(std::unique(v.begin(), v.end()), v.end()); }
    // blocks = connected components of the unknown graph; RCM inside each
    std::vector<int32_t> perm;       // new -> raw
    perm.reserve(nunk);
    std::vector<char> seen(nunk, 0);
    s->blk_off.assign(1, 0);
    for (int64_t r0 = 0; r0 < nunk; ++r0) {
        if (seen[r0]) continue;
        // component members
        std::vector<int32_t> comp{int32_t(r0)};
        seen[r0] = 1;
        for (size_t k = 0; k < comp.size(); ++k)
            for (int32_t w : uadj[comp[k]])
                if (!seen[w]) { seen[w] = 1; comp.push_back(w); }
        // pseudo-peripheral start: farthest node of two BFS sweeps, ties by lower degree
        auto bfs_far = [&](int32_t st) {
            std::map<int32_t, int32_t> dist;
            std::deque<int32_t> q{st};
            dist[st] = 0;
            int32_t far = st;
            while (!q.empty()) {
                int32_t u = q.front();
                q.pop_front();
                if (dist[u] > dist[far] || (dist[u] == dist[far] && uadj[u].size() < uadj[far].size())) far = u;
                for (int32_t w : uadj[u])
                    if (!dist.count(w)) { dist[w] = dist[u] + 1; q.push_back(w); }
            }
            return far;
        };
        int32_t start = bfs_far(bfs_far(comp[0]));
        std::vector<int32_t> order{start};
        std::map<int32_t, char> vis;
        vis[start] = 1;
        for (size_t k = 0; k < order.size(); ++k) {
            std::vector<int32_t> nbr;
            for (int32_t w : uadj[order[k]])
                if (!vis.count(w)) { vis[w] = 1; nbr.push_back(w); }
            std::sort(nbr.begin(), nbr.end(), [&](int32_t a, int32_t b) {
                return uadj[a].size() != uadj[b].size() ? uadj[a].size() < uadj[b].size() : a < b;
            });
            order.insert(order.end(), nbr.begin(), nbr.end());
        }
        std::reverse(order.begin(), order.end());
        perm.insert(perm.end(), order.begin(), order.end());
        s->blk_off.push_back(int64_t(perm.size()));
    }
    std::vector<int32_t> inv(nunk);
    for (int64_t i = 0; i < nunk; ++i) inv[perm[i]] = int32_t(i);
    int32_t W = 0;
    for (int64_t a = 0; a < nunk; ++a)
        for (int32_t b : uadj[a]) W = std::max<int32_t>(W, std::abs(inv[a] - inv[b]));
    s->W = std::max<int32_t>(W, 1);
    // nested dissection in place of the band when the band is too wide for the band
    // factorisation (or when asked for): unknowns placed at their nodes' centroids
    if (nunk > 0 && (p->pc_method == SIE_PC_ND || (p->pc_method == SIE_PC_AUTO && s->W >= kWideMax))) {
        std::vector<double> xyz(3 * size_t(nunk), 0.0);
        std::vector<int32_t> cnt(nunk, 0);
        for (int64_t t = 0; t < p->nt; ++t) {
            const int32_t u = unk_raw[L->node_of_tri[t]];
            if (u < 0) continue;
            for (int d = 0; d < 3; ++d) xyz[3 * size_t(u) + d] += p->tri_cen[3 * t + d];
            cnt[u]++;
        }
        for (int64_t u = 0; u < nunk; ++u)
            for (int d = 0; d < 3; ++d) xyz[3 * size_t(u) + d] /= std::max(cnt[u], 1);
        int rcn = nd_build(uadj, xyz, perm, &s->nd);
        if (rcn) return rcn;
        for (int64_t i = 0; i < nunk; ++i) inv[perm[i]] = int32_t(i);
        s->blk_off.assign({0, nunk});
    }
    std::vector<int32_t> unk(nn, -1);
    for (int64_t v = 0; v < nn; ++v) unk[v] = unk_raw[v] >= 0 ? inv[unk_raw[v]] : -1;
    // rows: incident branches of each unknown's member nodes
    std::vector<std::vector<std::pair<int32_t, int8_t>>> rows(nunk);
    for (int64_t e = 0; e < nb; ++e) {
        int32_t a = unk[L->tail[e]], b = unk[L->head[e]];
        if (a >= 0 && a != b) rows[a].emplace_back(int32_t(e), int8_t(1));
        if (b >= 0 && a != b) rows[b].emplace_back(int32_t(e), int8_t(-1));
    }
    std::vector<int32_t> row_ptr{0}, row_br, row_oth;
    std::vector<int8_t> row_sg;
    for (int64_t i = 0; i < nunk; ++i) {
        for (auto [e, sg] : rows[i]) {
            row_br.push_back(e);
            row_sg.push_back(sg);
            int32_t o = sg > 0 ? unk[L->head[e]] : unk[L->tail[e]];
            row_oth.push_back(o);
        }
        row_ptr.push_back(int32_t(row_br.size()));
    }
    if (s->nd) {
        int rcn = nd_rows(s->nd, row_ptr, row_oth);
        if (rcn) return rcn;
    }
    std::vector<int32_t> off_ptr{0}, off_port;
    std::vector<int8_t> off_sign;
    for (int64_t v = 0; v < nn; ++v) {
        for (auto [q, sg] : off[v]) { off_port.push_back(q); off_sign.push_back(sg); }
        off_ptr.push_back(int32_t(off_port.size()));
    }
    std::vector<int32_t> src_ptr{0}, src_br;
    std::vector<int8_t> src_sg;
    for (int64_t q = 0; q < np; ++q) {
        int32_t v = L->port_src[q];
        for (int64_t e = 0; e < nb; ++e) {
            if (L->tail[e] == v) { src_br.push_back(int32_t(e)); src_sg.push_back(1); }
            else if (L->head[e] == v) { src_br.push_back(int32_t(e)); src_sg.push_back(-1); }
        }
        src_ptr.push_back(int32_t(src_br.size()));
    }
    std::vector<int32_t> port_loop(std::max<int64_t>(np, 1), 0);
    for (int64_t q = 0; q < np; ++q) port_loop[q] = L->loop_of_branch[nb + q];
    std::vector<int64_t> bo(s->blk_off);
    s->tile_off.assign(1, 0);
    for (size_t k = 0; k + 1 < bo.size(); ++k) s->tile_off.push_back(s->tile_off.back() + (bo[k + 1] - bo[k] + 31) / 32);
    s->nchunks = s->tile_off.back();
    std::vector<int64_t> to(s->tile_off);
    int rc;
    if ((rc = pc_upload(s, &s->d_blk_off, bo))) return rc;
    if ((rc = pc_upload(s, &s->d_tile_off, to))) return rc;
    if ((rc = pc_upload(s, &s->d_unk_of_node, unk))) return rc;
    if ((rc = pc_upload(s, &s->d_off_ptr, off_ptr))) return rc;
    if ((rc = pc_upload(s, &s->d_off_port, off_port))) return rc;
    if ((rc = pc_upload(s, &s->d_off_sign, off_sign))) return rc;
    if ((rc = pc_upload(s, &s->d_row_ptr, row_ptr))) return rc;
    if ((rc = pc_upload(s, &s->d_row_br, row_br))) return rc;
    if ((rc = pc_upload(s, &s->d_row_sg, row_sg))) return rc;
    if ((rc = pc_upload(s, &s->d_row_oth, row_oth))) return rc;
    if ((rc = pc_upload(s, &s->d_src_ptr, src_ptr))) return rc;
    if ((rc = pc_upload(s, &s->d_src_br, src_br))) return rc;
    if ((rc = pc_upload(s, &s->d_src_sg, src_sg))) return rc;
    if ((rc = pc_upload(s, &s->d_port_loop, port_loop))) return rc;
    SIE_CUDA(cudaMalloc((void **)&s->d_status, sizeof(int)));
    s->allocs.push_back(s->d_status);
    return SIE_OK;
}

// FP64 complex values rounded to double-float pairs (k_round_cdf) or to FP32 (k_round_c)
__global__ void k_round_cdf(const double2 *__restrict__ a, cdf *__restrict__ b, int64_t n) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    b[i] = cdf{df(a[i].x), df(a[i].y)};
}
__global__ void k_round_c(const double2 *__restrict__ a, float2 *__restrict__ b, int64_t n) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2(float(a[i].x), float(a[i].y));
}

// 1/D_e with D_e = Z_s(sigma_e, w) G_ee + j w mu0/(4 pi) Lt_ee (Eq. Zb diagonal);
// Lt_ee is the static self term diag_L[e], or with the lossy kernel the complex
// per-frequency term diag_Lc[f][e] (diag_Lc NULL for the static kernel).
__global__ void k_pc_admittance(const double *__restrict__ diag_gram, const double *__restrict__ diag_L,
                                const double2 *__restrict__ diag_Lc, const int32_t *__restrict__ br_cond,
                                const double *__restrict__ zs_cl, int ncond, int64_t nb, int32_t nslots,
                                double2 *__restrict__ a) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nb * nslots) return;
    int64_t f = i / nb, e = i % nb;
    const double *cf = zs_cl + f * (2 * ncond + 1);   // (Re Z_s, Im Z_s) per conductor, then c_L / j
    const double zr = cf[2 * br_cond[e]], zi = cf[2 * br_cond[e] + 1], cl = cf[2 * ncond];
    const double2 L = diag_Lc ? diag_Lc[i] : make_double2(diag_L[e], 0.0);
    double dr = zr * diag_gram[e] - cl * L.y, di = zi * diag_gram[e] + cl * L.x;
    double den = dr * dr + di * di;
    a[i] = make_double2(dr / den, -di / den);
}

// Assemble the band of each (slot, block) and factorise it in place:
// K = L diag(d) L^T, unit L stored below the diagonal, d on the diagonal.
__global__ void __launch_bounds__(256) k_pc_factor(const int64_t *__restrict__ blk_off, int32_t nblk, int32_t W,
                                                   int64_t nunk, const int32_t *__restrict__ row_ptr,
                                                   const int32_t *__restrict__ row_br,
                                                   const int32_t *__restrict__ row_oth, const double2 *__restrict__ a,
                                                   int64_t nb, double2 *__restrict__ band, double2 *__restrict__ bandc,
                                                   int *status) {
    const int32_t f = blockIdx.x / nblk, b = blockIdx.x % nblk;
    const int64_t o = blk_off[b], n = blk_off[b + 1] - o;
    const int Wp = W + 1;
    double2 *B = band + (int64_t(f) * nunk + o) * Wp;
    double2 *Bc = bandc + (int64_t(f) * nunk + o) * Wp;
    const double2 *af = a + int64_t(f) * nb;
    for (int64_t i = threadIdx.x; i < n * Wp; i += blockDim.x) B[i] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t gi = o + i;
        double2 d = make_double2(0.0, 0.0);
        for (int32_t k = row_ptr[gi]; k < row_ptr[gi + 1]; ++k) {
            double2 w = af[row_br[k]];
            d = cadd(d, w);
            int32_t j = row_oth[k];
            if (j >= 0 && j < gi) {   // lower triangle entry (i, j): K_ij -= a_e
                int64_t dd = gi - j;
                B[i * Wp + dd] = csub(B[i * Wp + dd], w);
            }
        }
        B[i * Wp] = d;
    }
    __syncthreads();
    // pivot column staged per step: kc[r] = K[k+r][k], lc[r] = K[k+r][k] / d_k (r = 1..W)
    __shared__ double2 kc[kWideMax], lc[kWideMax];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 tile over (row, column)
    for (int64_t k = 0; k < n; ++k) {
        const double2 dk = B[k * Wp];
        if (dk.x == 0.0 && dk.y == 0.0) {
            if (threadIdx.x == 0) *status = SIE_ERR_BREAKDOWN;
            return;
        }
        const double den = dk.x * dk.x + dk.y * dk.y;
        const double2 inv = make_double2(dk.x / den, -dk.y / den);
        const int m = int((int64_t(W) < n - 1 - k) ? int64_t(W) : n - 1 - k);
        // rows i = k + r (r = 1..m): K[i][k+c] -= l_ik d_k l_(k+c)k for c in 1..r; the
        // pivot column (offset r of row k + r) is never written by the update itself
        if (W < kWideMax) {
            for (int r = 1 + threadIdx.x; r <= m; r += blockDim.x) {
                const double2 v = B[(k + r) * Wp + r];
                kc[r] = v;
                lc[r] = cmul(v, inv);
            }
            __syncthreads();
            for (int r = 1 + ty; r <= m; r += 16) {
                const double2 lr = lc[r];
                double2 *row = B + (k + r) * Wp + r;       // row[-c] = K[k+r][k+c]
                for (int c = 1 + tx; c <= r; c += 16) row[-c] = csub(row[-c], cmul(lr, kc[c]));
            }
            for (int r = 1 + threadIdx.x; r <= m; r += blockDim.x) B[(k + r) * Wp + r] = lc[r];   // l_{k+r,k}
        } else {   // bands too wide to stage the column: read it where it is
            for (int r = 1 + ty; r <= m; r += 16) {
                const double2 lr = cmul(B[(k + r) * Wp + r], inv);
                double2 *row = B + (k + r) * Wp + r;
                for (int c = 1 + tx; c <= r; c += 16) row[-c] = csub(row[-c], cmul(lr, B[(k + c) * Wp + c]));
            }
            __syncthreads();
            for (int r = 1 + threadIdx.x; r <= m; r += blockDim.x)
                B[(k + r) * Wp + r] = cmul(B[(k + r) * Wp + r], inv);
        }
        __syncthreads();
    }
    // column-major copy for the forward sweep: Bc[i][d] = L[i+d][i], Bc[i][0] = d_i
    for (int64_t t = threadIdx.x; t < n * Wp; t += blockDim.x) {
        const int64_t i = t / Wp, d = t % Wp;
        Bc[t] = d == 0 ? B[i * Wp] : (i + d < n ? B[(i + d) * Wp + d] : make_double2(0.0, 0.0));
    }
}

// Drive of each branch: kappa_e = a_e (off_tail - off_head + emf_e), emf on links.
// T = float (mixed form): the preconditioner is an approximation of P, so its
// bookkeeping runs in FP32 like its band factors.
template <typename T>
__global__ void k_pc_drive(const double2 *__restrict__ y, int64_t nl, const C<T> *__restrict__ a,
                           const int32_t *__restrict__ slot, const int32_t *__restrict__ loop_of_branch,
                           const int32_t *__restrict__ tail, const int32_t *__restrict__ head,
                           const int32_t *__restrict__ off_ptr, const int32_t *__restrict__ off_port,
                           const int8_t *__restrict__ off_sign, const int32_t *__restrict__ port_loop, int64_t nb,
                           int32_t nrhs, C<T> *__restrict__ kappa) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nb * nrhs) return;
    int64_t r = i / nb, e = i % nb;
    const double2 *yr = y + r * nl;
    auto ld = [&](int64_t k) { const double2 q = yr[k]; return mk<T>(T(q.x), T(q.y)); };
    C<T> v = mk<T>(T(0), T(0));
    int32_t l = loop_of_branch[e];
    if (l >= 0) v = ld(l);
    int32_t t = tail[e], h = head[e];
    for (int32_t k = off_ptr[t]; k < off_ptr[t + 1]; ++k) {
        const C<T> q = ld(port_loop[off_port[k]]);
        v = off_sign[k] > 0 ? cadd(v, q) : csub(v, q);
    }
    for (int32_t k = off_ptr[h]; k < off_ptr[h + 1]; ++k) {
        const C<T> q = ld(port_loop[off_port[k]]);
        v = off_sign[k] > 0 ? csub(v, q) : cadd(v, q);
    }
    kappa[i] = cmul(a[int64_t(slot[r]) * nb + e], v);
}

// rhs_i = -sum over incident branches of s * kappa_e; then band solve
// L d L^T u = rhs per (rhs, block) on one warp.
__global__ void k_pc_solve(const double2 *__restrict__ kappa, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ row_br, const int8_t *__restrict__ row_sg,
                           const int64_t *__restrict__ blk_off, int32_t nblk, int32_t W, int64_t nunk, int64_t nb,
                           const double2 *__restrict__ band, const int32_t *__restrict__ slot, int32_t nrhs,
                           double2 *__restrict__ u) {
    const int64_t wid = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (wid >= int64_t(nrhs) * nblk) return;
    const int64_t r = wid / nblk, b = wid % nblk;
    const int64_t o = blk_off[b], n = blk_off[b + 1] - o;
    const int Wp = W + 1;
    const double2 *B = band + (int64_t(slot[r]) * nunk + o) * Wp;
    double2 *x = u + r * nunk + o;
    const double2 *kr = kappa + r * nb;
    for (int64_t i = lane; i < n; i += 32) {
        double2 acc = make_double2(0.0, 0.0);
        for (int32_t k = row_ptr[o + i]; k < row_ptr[o + i + 1]; ++k)
            acc = row_sg[k] > 0 ? csub(acc, kr[row_br[k]]) : cadd(acc, kr[row_br[k]]);
        x[i] = acc;
    }
    __syncwarp();
    // forward: x_i -= sum_{d=1..W} L[i][i-d] x_{i-d}
    for (int64_t i = 0; i < n; ++i) {
        double2 acc = make_double2(0.0, 0.0);
        for (int d = 1 + lane; d <= W; d += 32)
            if (i - d >= 0) acc = cadd(acc, cmul(B[i * Wp + d], x[i - d]));
        for (int s = 16; s > 0; s >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, s);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, s);
        }
        if (lane == 0) x[i] = csub(x[i], acc);
        __syncwarp();
    }
    for (int64_t i = lane; i < n; i += 32) {
        double2 d = B[i * Wp];
        double den = d.x * d.x + d.y * d.y;
        x[i] = cmul(x[i], make_double2(d.x / den, -d.y / den));
    }
    __syncwarp();
    // backward: x_i -= sum_{d=1..W} L[i+d][d] x_{i+d}
    for (int64_t i = n - 1; i >= 0; --i) {
        double2 acc = make_double2(0.0, 0.0);
        for (int d = 1 + lane; d <= W; d += 32)
            if (i + d < n) acc = cadd(acc, cmul(B[(i + d) * Wp + d], x[i + d]));
        for (int s = 16; s > 0; s >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, s);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, s);
        }
        if (lane == 0) x[i] = csub(x[i], acc);
        __syncwarp();
    }
}

// Band solve L d L^T u = rhs for bands wider than a warp (31 < W < 1024), one
// CTA of Wt >= W threads per (right-hand side, block), after assembling
// rhs_i = -sum over the incident branches of s * kappa_e.  The sweeps go 32 pivots at a time: the CTA
// stages the chunk's 32 x 32 triangle of L in shared memory, warp 0 finishes the
// chunk's rows in registers (a shuffle broadcasts each pivot, no CTA barrier),
// then every thread subtracts the chunk's contribution from one of the W band
// rows below (32 consecutive entries of its row of the band: the row-major band
// in the forward sweep, the column-major copy in the backward sweep), and the
// rows that enter the band take their right-hand sides.  Pending values live in
// a circular shared-memory window of S >= W + 32 rows.  Three barriers per 32
// pivots instead of one per pivot.
template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT) k_pc_sweep_blk(
    const C<T> *__restrict__ kappa, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ row_br,
    const int8_t *__restrict__ row_sg, const int64_t *__restrict__ blk_off, int32_t nblk, int32_t W, int32_t S,
    int64_t nunk, int64_t nb, const C<T> *__restrict__ band, const C<T> *__restrict__ bandc,
    const int32_t *__restrict__ slot, C<T> *__restrict__ u) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T> *pend = reinterpret_cast<C<T> *>(smem_raw);   // [S] window of pending rows
    C<T> *tri = pend + S;                              // [32][33] chunk triangle
    C<T> *xc = tri + 32 * 33;                          // [32] finished chunk values
    const int64_t r = blockIdx.x / nblk, b = blockIdx.x % nblk;
    const int64_t o = blk_off[b], n = blk_off[b + 1] - o;
    const int Wp = W + 1, nt = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    const C<T> *B = band + (int64_t(slot[r]) * nunk + o) * Wp;
    const C<T> *Bc = bandc + (int64_t(slot[r]) * nunk + o) * Wp;
    C<T> *x = u + r * nunk + o;
    const C<T> *kr = kappa + r * nb;
    const C<T> zero = mk<T>(T(0), T(0));
    const int64_t smask = S - 1;
    for (int64_t i = tid; i < n; i += nt) {
        C<T> acc = zero;
        for (int32_t k = row_ptr[o + i]; k < row_ptr[o + i + 1]; ++k)
            acc = row_sg[k] > 0 ? csub(acc, kr[row_br[k]]) : cadd(acc, kr[row_br[k]]);
        x[i] = acc;
    }
    __syncthreads();
    // ---- forward: L z = rhs, rows in increasing order
    for (int64_t i = tid; i < n && i < W + 32; i += nt) pend[i & smask] = x[i];
    for (int64_t k0 = 0; k0 < n; k0 += 32) {
        __syncthreads();                               // window rows of this chunk are final
#pragma unroll 8
        for (int e = tid; e < 32 * 32; e += nt) {      // tri[l][j] = L[k0+l][k0+j], j < l
            const int l = e >> 5, j = e & 31;
            tri[l * 33 + j] = (j < l && k0 + l < n) ? B[(k0 + l) * Wp + (l - j)] : zero;
        }
        __syncthreads();
        if (tid < 32) {
            C<T> v = k0 + lane < n ? pend[(k0 + lane) & smask] : zero;
#pragma unroll 4
            for (int j = 0; j < 31; ++j) {
                C<T> xj;
                xj.x = __shfl_sync(0xffffffffu, v.x, j);
                xj.y = __shfl_sync(0xffffffffu, v.y, j);
                if (lane > j) v = csub(v, cmul(tri[lane * 33 + j], xj));
            }
            xc[lane] = v;
            if (k0 + lane < n) x[k0 + lane] = v;
        }
        __syncthreads();
        // rows k0 + 32 + t (t < W) take the chunk's contribution; rows entering the band take rhs
        for (int t = tid; t < W; t += nt) {
            const int64_t i = k0 + 32 + t;
            if (i >= n) break;
            const C<T> *row = B + i * Wp;              // L[i][k0+j] = row[32 + t - j]
            const int j0 = 32 + t - W > 0 ? 32 + t - W : 0;   // band edge
            // loads issued in batches of KB ahead of their multiply-adds (KB = 32 where the
            // register budget allows, 8 under the 1024-thread cap)
            constexpr int KB = MAXT > 256 ? 8 : 32;
            C<T> acc = zero;
#pragma unroll
            for (int jb = 0; jb < 32; jb += KB) {
                C<T> e[KB];
#pragma unroll
                for (int q = 0; q < KB; ++q) e[q] = row[jb + q >= j0 ? 32 + t - jb - q : 32 + t - 31];
#pragma unroll
                for (int q = 0; q < KB; ++q)
                    if (jb + q >= j0) acc = cadd(acc, cmul(e[q], xc[jb + q]));
            }
            pend[i & smask] = csub(pend[i & smask], acc);
        }
        for (int t = tid; t < 32; t += nt) {
            const int64_t i = k0 + 32 + W + t;
            if (i < n) pend[i & smask] = x[i];
        }
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += nt) {           // diagonal: x_i /= d_i
        const C<T> dg = B[i * Wp];
        const T den = dg.x * dg.x + dg.y * dg.y;
        x[i] = cmul(x[i], mk<T>(dg.x / den, -dg.y / den));
    }
    __syncthreads();
    // ---- backward: L^T u = z, rows in decreasing order; row q = n - 1 - k in the window
    for (int64_t k = tid; k < n && k < W + 32; k += nt) pend[k & smask] = x[n - 1 - k];
    for (int64_t k0 = 0; k0 < n; k0 += 32) {
        __syncthreads();
        const int64_t k1 = n - 1 - k0;                 // the chunk's top row
#pragma unroll 8
        for (int e = tid; e < 32 * 32; e += nt) {      // tri[l][j] = L[k1-j][k1-l], j < l
            const int l = e >> 5, j = e & 31;
            tri[l * 33 + j] = (j < l && k0 + l < n) ? Bc[(k1 - l) * Wp + (l - j)] : zero;
        }
        __syncthreads();
        if (tid < 32) {
            C<T> v = k0 + lane < n ? pend[(k0 + lane) & smask] : zero;
#pragma unroll 4
            for (int j = 0; j < 31; ++j) {
                C<T> xj;
                xj.x = __shfl_sync(0xffffffffu, v.x, j);
                xj.y = __shfl_sync(0xffffffffu, v.y, j);
                if (lane > j) v = csub(v, cmul(tri[lane * 33 + j], xj));
            }
            xc[lane] = v;
            if (k0 + lane < n) x[k1 - lane] = v;
        }
        __syncthreads();
        for (int t = tid; t < W; t += nt) {
            const int64_t k = k0 + 32 + t;             // row k1 - 32 - t
            if (k >= n) break;
            const C<T> *col = Bc + (n - 1 - k) * Wp;   // L[k1-j][row] = col[32 + t - j]
            const int j0 = 32 + t - W > 0 ? 32 + t - W : 0;
            // loads issued in batches of KB ahead of their multiply-adds (KB = 32 where the
            // register budget allows, 8 under the 1024-thread cap)
            constexpr int KB = MAXT > 256 ? 8 : 32;
            C<T> acc = zero;
#pragma unroll
            for (int jb = 0; jb < 32; jb += KB) {
                C<T> e[KB];
#pragma unroll
                for (int q = 0; q < KB; ++q) e[q] = col[jb + q >= j0 ? 32 + t - jb - q : 32 + t - 31];
#pragma unroll
                for (int q = 0; q < KB; ++q)
                    if (jb + q >= j0) acc = cadd(acc, cmul(e[q], xc[jb + q]));
            }
            pend[k & smask] = csub(pend[k & smask], acc);
        }
        for (int t = tid; t < 32; t += nt) {
            const int64_t k = k0 + 32 + W + t;
            if (k < n) pend[k & smask] = x[n - 1 - k];
        }
    }
}

// Same solve with the band sweeps kept in registers (requires W <= 31): lane
// (row mod 32) holds the running value of `row` for the 32 rows from the current
// pivot on.  A step broadcasts the finished pivot with one shuffle and each lane
// applies one multiply-add; the pivot's lane then takes the row 32 further on.
template <typename V> __device__ __forceinline__ V shfl_c(V v, int src) {
    v.x = shfl1(v.x, src);
    v.y = shfl1(v.y, src);
    return v;
}

// Band solve L d L^T u = rhs of one conductor block for one right-hand side,
// one warp (requires W <= 31), in place on the right-hand sides k_pc_rhs
// assembled (rhs_i = -sum over the incident branches of s * kappa_e).
//
// The sweeps keep a circular window in registers: lane (row mod 32) holds the
// running value of its row for the 32 rows from the current pivot on.  A step
// broadcasts the finished pivot with a shuffle, every lane subtracts its band
// entry times the pivot, and the pivot's lane takes over the row 32 further
// on.  The band entries come from sweep tiles built with the factor: per chunk
// of 32 pivots, tile[lane][step] (pitch 33) is the entry lane `lane` applies at
// step `step` (zero where it has none), so a step reads its entry with one
// shared-memory load at a fixed offset, conflict-free, and no index
// arithmetic.  Each warp keeps pc_nbuf tile buffers; the tile of chunk c + NB
// is requested as soon as chunk c is done.
constexpr int PC_CH = 32;
constexpr int PC_TP = 33;                          // tile pitch (complex)
constexpr int PC_TILE = PC_CH * PC_TP;             // complex per tile

// tiles[slot][dir][chunk][lane][PC_TP]: dir 0 forward (entries of L below the
// pivot, from bandc), dir 1 backward (from band); chunk c of block b covers
// pivots 32 c .. 32 c + 31 (forward) or n-1-32c .. n-32-32c (backward).
template <typename T>
__global__ void k_pc_tiles(const double2 *__restrict__ band, const double2 *__restrict__ bandc,
                           const int64_t *__restrict__ blk_off, const int64_t *__restrict__ tile_off, int32_t nblk,
                           int32_t W, int64_t nunk, int64_t nchunks, int32_t ns, C<T> *__restrict__ tiles) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t per = nchunks * PC_TILE;
    if (i >= int64_t(ns) * 2 * per) return;
    const int j = int(i % PC_TP);
    int64_t t = i / PC_TP;
    const int L = int(t % PC_CH);
    t /= PC_CH;
    const int64_t gc = t % nchunks;
    t /= nchunks;
    const int dir = int(t % 2);
    const int64_t s = t / 2;
    int lo = 0, hi = nblk - 1;   // block holding chunk gc: tile_off[b] <= gc < tile_off[b + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (tile_off[mid] <= gc) lo = mid; else hi = mid - 1;
    }
    const int64_t c = gc - tile_off[lo], o = blk_off[lo], n = blk_off[lo + 1] - o;
    C<T> v = mk<T>(T(0), T(0));
    if (j < PC_CH) {
        const int d = (L - j) & 31;
        const int64_t row = dir == 0 ? PC_CH * c + j : n - 1 - PC_CH * c - j;
        const bool ok = d >= 1 && d <= W && row >= 0 && row < n && (dir == 0 ? row + d < n : row - d >= 0);
        if (ok) {
            const double2 e = (dir == 0 ? bandc : band)[(s * nunk + o + row) * (W + 1) + d];
            v = mk<T>(T(e.x), T(e.y));
        }
    }
    tiles[i] = v;
}

// dinv[slot][i] = 1 / d_i, the reciprocal pivots of the LDL^T factor (FP64, rounded to T).
template <typename T>
__global__ void k_pc_dinv(const double2 *__restrict__ band, int64_t total, int32_t Wp, C<T> *__restrict__ dinv) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const double2 d = band[i * Wp];
    const double den = d.x * d.x + d.y * d.y;
    dinv[i] = mk<T>(T(d.x / den), T(-d.y / den));
}

// copy one tile into shared memory with 16-byte asynchronous copies
template <typename T>
__device__ __forceinline__ void pc_stage_tile(C<T> *dst, const C<T> *src, int lane) {
    constexpr int n16 = PC_TILE * int(sizeof(C<T>)) / 16;
    const unsigned s0 = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    const char *g = reinterpret_cast<const char *>(src);
    for (int k = lane; k < n16; k += 32)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s0 + 16u * unsigned(k)), "l"(g + 16 * k));
}

// One step of a sweep: pivot j of the chunk; tl = this lane's tile row.  The
// update w - l xi is fused (four FMAs); the pivot's lane keeps xi and takes pf.
// t is every lane's updated value before that hand-over.  The pivot lane of the
// next step was not this step's pivot, so its t equals its w, and the broadcast
// reads t: the select stays off the chain from one pivot to the next.
// Double-float step, t = w - l xi with the pivot-to-pivot chain on the high
// parts only: hi = (w.hi + p1) + p2 with p1, p2 the FP32 products of the high
// parts (two FP32 operations deep), and every rounding error of those products
// (two-product) and sums (two-sum), the low-part products and w.lo collected in
// lo, which is added last and which no later high part waits for.  The pair
// stays unnormalised during the sweep: a row takes at most W <= 31 updates
// before it is a pivot, so lo stays a few units of hi's last place and hi + lo
// carries about 48 bits; the stores normalise it.
__device__ __forceinline__ float tprod(float a, float b, float &e) {
    const float p = a * b;
    e = fmaf(a, b, -p);
    return p;
}
__device__ __forceinline__ float tsum(float a, float b, float &e) {
    const float s = a + b, bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}
// w - (a1 x1 + a2 x2) with (a, x) double-float pairs, the high-part chain two deep
__device__ __forceinline__ df df_sub2(df w, df a1, df x1, df a2, df x2) {
    float e1, e2, f1, f2;
    const float p1 = tprod(-a1.hi, x1.hi, e1), p2 = tprod(-a2.hi, x2.hi, e2);
    const float s1 = tsum(w.hi, p1, f1), s2 = tsum(s1, p2, f2);
    float lo = (((w.lo + e1) + e2) + (f1 + f2));
    lo = fmaf(-a1.lo, x1.hi, lo);
    lo = fmaf(-a2.lo, x2.hi, lo);
    lo = fmaf(-a1.hi, x1.lo, lo);
    lo = fmaf(-a2.hi, x2.lo, lo);
    return df(s2, lo);
}

template <typename T>
__device__ __forceinline__ void pc_step(const C<T> *tl, int j, int lane, C<T> &w, C<T> &t, const C<T> &pf,
                                        C<T> &done) {
    const C<T> l = tl[j];
    const C<T> xi = shfl_c(t, j);
    if constexpr (std::is_same<T, df>::value) {
        // re: w.re - (l.re xi.re - l.im xi.im), im: w.im - (l.re xi.im + l.im xi.re)
        t.x = df_sub2(w.x, l.x, xi.x, -l.y, xi.y);
        t.y = df_sub2(w.y, l.x, xi.y, l.y, xi.x);
        const bool me = lane == j;
        done.x = me ? xi.x : done.x;
        done.y = me ? xi.y : done.y;
        w.x = me ? pf.x : t.x;
        w.y = me ? pf.y : t.y;
        return;
    }
    t.x = fma(-l.x, xi.x, fma(l.y, xi.y, w.x));
    t.y = fma(-l.x, xi.y, fma(-l.y, xi.x, w.y));
    const bool me = lane == j;
    done.x = me ? xi.x : done.x;
    done.y = me ? xi.y : done.y;
    w.x = me ? pf.x : t.x;
    w.y = me ? pf.y : t.y;
}
// the 32 steps of a full chunk, unrolled at compile time
template <typename T, int J>
__device__ __forceinline__ void pc_chunk(const C<T> *tl, int lane, C<T> &w, C<T> &t, const C<T> &pf, C<T> &done) {
    if constexpr (J < PC_CH) {
        pc_step<T>(tl, J, lane, w, t, pf, done);
        pc_chunk<T, J + 1>(tl, lane, w, t, pf, done);
    }
}

// Right-hand sides of the nodal systems, rhs_i = -sum over the incident
// branches e of s * kappa_e (s = +-1), one thread per (right-hand side, row),
// branches in their stored order.  Run as its own fully occupied kernel: inside
// the sweep kernel, at one warp per (right-hand side, block), its chains of
// dependent gathers were exposed.
template <typename T>
__global__ void k_pc_rhs(const C<T> *__restrict__ kappa, const int32_t *__restrict__ row_ptr,
                         const int32_t *__restrict__ row_br, const int8_t *__restrict__ row_sg, int64_t nunk,
                         int64_t nb, int32_t R, C<T> *__restrict__ xs) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= int64_t(R) * nunk) return;
    const int64_t r = g / nunk, row = g - r * nunk;
    const C<T> *kr = kappa + r * nb;
    C<T> acc = mk<T>(T(0), T(0));
    for (int32_t q = row_ptr[row]; q < row_ptr[row + 1]; ++q)
        acc = row_sg[q] > 0 ? csub(acc, kr[row_br[q]]) : cadd(acc, kr[row_br[q]]);
    xs[g] = acc;
}

// Tile buffers per warp in the sweep kernel: tiles are fetched NBUF - 1 chunks
// ahead of their use.
template <typename T> __host__ __device__ constexpr int pc_nbuf() { return sizeof(T) == 4 ? 3 : 2; }

template <typename T>
__global__ void __launch_bounds__(128, 2) k_pc_sweep(
    const int64_t *__restrict__ blk_off, const int64_t *__restrict__ tile_off, int32_t nblk, int64_t nunk,
    int64_t nchunks, const C<T> *__restrict__ tiles, const C<T> *__restrict__ dinv, const int32_t *__restrict__ slot,
    int32_t R, C<T> *__restrict__ xs) {
    constexpr int NB = pc_nbuf<T>();
    extern __shared__ __align__(16) unsigned char pc_smem[];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t wid = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (wid >= int64_t(R) * nblk) return;
    const int32_t r = int32_t(wid / nblk), b = int32_t(wid % nblk);
    const int64_t o = blk_off[b], n = blk_off[b + 1] - o;
    const int64_t sl = slot[r];
    const C<T> *Tf = tiles + ((sl * 2 + 0) * nchunks + tile_off[b]) * PC_TILE;
    const C<T> *Tb = tiles + ((sl * 2 + 1) * nchunks + tile_off[b]) * PC_TILE;
    const C<T> *dv = dinv + sl * nunk + o;
    const C<T> zero = mk<T>(T(0), T(0));
    C<T> *buf = reinterpret_cast<C<T> *>(pc_smem) + int64_t(wl) * NB * PC_TILE;   // [warp][NB][PC_TILE]
    C<T> *x = xs + int64_t(r) * nunk + o;
    const int64_t nch = (n + PC_CH - 1) / PC_CH;
    // the first NB tiles in flight; one commit group per chunk, so that at chunk
    // c at most NB - 1 groups (those of chunks c + 1 .. c + NB - 1) may pend
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if (k < nch) pc_stage_tile<T>(buf + k * PC_TILE, Tf + k * PC_TILE, lane);
        asm volatile("cp.async.commit_group;\n" ::);
    }
    // ---------------- forward: y_{i+d} -= L[i+d][i] y_i, then y_i /= d_i at the store
    C<T> w = lane < n ? x[lane] : zero, pf = lane + 32 < n ? x[lane + 32] : zero, done = zero, t = w;
    int bs = 0;   // buffer of chunk c: c mod NB
    for (int64_t c = 0; c < nch; ++c) {
        const int64_t base = c * PC_CH;
        const C<T> pn = base + 64 + lane < n ? x[base + 64 + lane] : zero;   // row taken over in chunk c + 1
        const C<T> di = base + lane < n ? dv[base + lane] : zero;
        asm volatile("cp.async.wait_group %0;\n" ::"n"(NB - 1));
        __syncwarp();
        const C<T> *tl = buf + bs * PC_TILE + lane * PC_TP;
        if (base + PC_CH <= n) {
            pc_chunk<T, 0>(tl, lane, w, t, pf, done);
        } else {
            for (int j = 0; j < int(n - base); ++j) pc_step<T>(tl, j, lane, w, t, pf, done);
        }
        if (base + lane < n) x[base + lane] = cmul(done, di);
        pf = pn;
        __syncwarp();
        if (c + NB < nch) pc_stage_tile<T>(buf + bs * PC_TILE, Tf + (c + NB) * PC_TILE, lane);
        asm volatile("cp.async.commit_group;\n" ::);
        bs = bs + 1 == NB ? 0 : bs + 1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncwarp();
    // ---------------- backward: x_{i-d} -= L[i][i-d] x_i   (chunk c = pivots i = n-1-32c-j)
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        if (k < nch) pc_stage_tile<T>(buf + k * PC_TILE, Tb + k * PC_TILE, lane);
        asm volatile("cp.async.commit_group;\n" ::);
    }
    w = n - 1 - lane >= 0 ? x[n - 1 - lane] : zero;
    pf = n - 33 - lane >= 0 ? x[n - 33 - lane] : zero;
    done = zero;
    t = w;
    bs = 0;
    for (int64_t c = 0; c < nch; ++c) {
        const int64_t top = n - 1 - c * PC_CH;          // pivot of step j = 0
        const C<T> pn = top - 64 - lane >= 0 ? x[top - 64 - lane] : zero;
        asm volatile("cp.async.wait_group %0;\n" ::"n"(NB - 1));
        __syncwarp();
        const C<T> *tl = buf + bs * PC_TILE + lane * PC_TP;
        if (top - (PC_CH - 1) >= 0) {
            pc_chunk<T, 0>(tl, lane, w, t, pf, done);
        } else {
            for (int j = 0; j <= int(top); ++j) pc_step<T>(tl, j, lane, w, t, pf, done);
        }
        if (top - lane >= 0) x[top - lane] = done;   // final values in place (every row still to be read lies below)
        pf = pn;
        __syncwarp();
        if (c + NB < nch) pc_stage_tile<T>(buf + bs * PC_TILE, Tb + (c + NB) * PC_TILE, lane);
        asm volatile("cp.async.commit_group;\n" ::);
        bs = bs + 1 == NB ? 0 : bs + 1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}

// Branch currents i_e = a_e (phi_tail - phi_head + emf_e) = a_e (u_t - u_h) + kappa_e.
template <typename T>
__global__ void k_pc_currents(const C<T> *__restrict__ u, int64_t nunk, const C<T> *__restrict__ kappa,
                              const C<T> *__restrict__ a, const int32_t *__restrict__ slot,
                              const int32_t *__restrict__ unk, const int32_t *__restrict__ tail,
                              const int32_t *__restrict__ head, int64_t nb, int32_t nrhs, C<T> *__restrict__ ibr) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nb * nrhs) return;
    int64_t r = i / nb, e = i % nb;
    int32_t ut = unk[tail[e]], uh = unk[head[e]];
    C<T> d = mk<T>(T(0), T(0));
    if (ut >= 0) d = cadd(d, u[r * nunk + ut]);
    if (uh >= 0) d = csub(d, u[r * nunk + uh]);
    ibr[i] = cadd(cmul(a[int64_t(slot[r]) * nb + e], d), kappa[i]);
}

template <typename T>
__global__ void k_pc_out(const C<T> *__restrict__ ibr, const int32_t *__restrict__ link_branch,
                         const int32_t *__restrict__ src_ptr, const int32_t *__restrict__ src_br,
                         const int8_t *__restrict__ src_sg, int64_t nb, int64_t nl, int32_t nrhs,
                         double2 *__restrict__ z) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nl * nrhs) return;
    int64_t r = i / nl, l = i % nl;
    int32_t e = link_branch[l];
    const C<T> *ir = ibr + r * nb;
    C<T> v;
    if (e < nb) {
        v = ir[e];
    } else {
        int32_t q = int32_t(e - nb);
        v = mk<T>(T(0), T(0));
        for (int32_t k = src_ptr[q]; k < src_ptr[q + 1]; ++k)
            v = src_sg[k] > 0 ? cadd(v, ir[src_br[k]]) : csub(v, ir[src_br[k]]);
    }
    z[i] = make_double2(to_f64(v.x), to_f64(v.y));
}

inline unsigned nblk_(int64_t n, int t = 256) { return unsigned((n + t - 1) / t); }

// Factor slots for the distinct omegas of a right-hand-side batch.
int pc_prepare(pfft_plan *p, const double *omega, int32_t R, std::vector<int32_t> &slot, cudaStream_t st) {
    if (!p->pc) {
        int rc = build_symbolic(p);
        if (rc) { plan_free_precond(p); return rc; }
    }
    PrecondState *s = p->pc;
    std::vector<double> uniq(omega, omega + R);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    for (double w : uniq)
        if (!(w > 0.0 || (w == 0.0 && dc_defined(p))) || !std::isfinite(w))
            return fail(SIE_ERR_ARG, "preconditioner: omega must be positive (or 0 with a slab surface model on "
                                     "every conductor)");
    slot.resize(R);
    for (int32_t r = 0; r < R; ++r) slot[r] = int32_t(std::lower_bound(uniq.begin(), uniq.end(), omega[r]) - uniq.begin());
    if (R > s->cap_rhs) {
        for (void *a : {(void *)s->d_kappa, (void *)s->d_u, (void *)s->d_ibr, (void *)s->d_slot})
            if (a) cudaFreeAsync(a, st);
        s->d_kappa = s->d_u = s->d_ibr = nullptr;
        s->d_slot = nullptr;
        SIE_CUDA(pool_alloc(p, &s->d_kappa, size_t(R) * p->nb * sizeof(double2), st));
        SIE_CUDA(pool_alloc(p, &s->d_ibr, size_t(R) * p->nb * sizeof(double2), st));
        SIE_CUDA(pool_alloc(p, &s->d_u, size_t(R) * std::max<int64_t>(s->nunk, 1) * sizeof(double2), st));
        if (s->d_u32) cudaFreeAsync(s->d_u32, st);
        SIE_CUDA(pool_alloc(p, &s->d_u32, size_t(R) * std::max<int64_t>(s->nunk, 1) * sizeof(float2), st));
        SIE_CUDA(pool_alloc(p, &s->d_slot, size_t(R) * sizeof(int32_t), st));
        if (s->nd) {
            if (s->d_uv) cudaFreeAsync(s->d_uv, st);
            SIE_CUDA(pool_alloc(p, &s->d_uv, size_t(R) * std::max<int64_t>(nd_update_size(s->nd), 1) * sizeof(double2), st));
        }
        s->cap_rhs = R;
    }
    SIE_CUDA(cudaMemcpyAsync(s->d_slot, slot.data(), R * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (s->nd) {
        // the nested-dissection solves take the right-hand sides of one slot in groups
        const int G = nd_group_size();
        std::vector<int32_t> grp;
        for (int32_t f = 0; f < int32_t(uniq.size()); ++f) {
            std::vector<int32_t> rs;
            for (int32_t r = 0; r < R; ++r)
                if (slot[r] == f) rs.push_back(r);
            for (size_t k = 0; k < rs.size(); k += G)
                for (int g = 0; g < G; ++g) grp.push_back(k + g < rs.size() ? rs[k + g] : -1);
        }
        const int32_t ng = int32_t(grp.size() / G);
        if (ng > s->cap_grp) {
            if (s->d_grp) cudaFreeAsync(s->d_grp, st);
            s->d_grp = nullptr;
            SIE_CUDA(pool_alloc(p, &s->d_grp, grp.size() * sizeof(int32_t), st));
            s->cap_grp = ng;
        }
        SIE_CUDA(cudaMemcpyAsync(s->d_grp, grp.data(), grp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        SIE_CUDA(cudaStreamSynchronize(st));   // grp is a host temporary
        s->ngrp = ng;
    }
    if (uniq == s->slot_omega) return SIE_OK;   // factors cached
    const int32_t ns = int32_t(uniq.size());
    if (s->d_band) cudaFreeAsync(s->d_band, st);
    if (s->d_bandc) cudaFreeAsync(s->d_bandc, st);
    for (void *q : {(void *)s->d_tile64, (void *)s->d_dinv64, (void *)s->d_tile32, (void *)s->d_dinv32,
                    (void *)s->d_tiledf, (void *)s->d_dinvdf, (void *)s->d_adf})
        if (q) cudaFreeAsync(q, st);
    s->d_tile64 = s->d_dinv64 = nullptr;
    s->d_tile32 = s->d_dinv32 = nullptr;
    s->d_tiledf = s->d_dinvdf = nullptr;
    s->d_adf = nullptr;
    if (s->d_a) cudaFreeAsync(s->d_a, st);
    if (s->d_a32) cudaFreeAsync(s->d_a32, st);
    if (s->d_band32) cudaFreeAsync(s->d_band32, st);
    if (s->d_bandc32) cudaFreeAsync(s->d_bandc32, st);
    s->d_band32 = s->d_bandc32 = nullptr;
    s->d_band = nullptr;
    s->d_bandc = nullptr;
    s->d_a = nullptr;
    s->d_a32 = nullptr;
    s->slot_omega.clear();
    if (s->d_ndL64) cudaFreeAsync(s->d_ndL64, st);
    if (s->d_ndL32) cudaFreeAsync(s->d_ndL32, st);
    s->d_ndL64 = nullptr;
    s->d_ndL32 = nullptr;
    if (s->nd) {
        SIE_CUDA(pool_alloc(p, &s->d_ndL64, size_t(ns) * std::max<int64_t>(nd_factor_size(s->nd), 1) * sizeof(double2), st));
        SIE_CUDA(pool_alloc(p, &s->d_ndL32, size_t(ns) * std::max<int64_t>(nd_factor_size(s->nd), 1) * sizeof(float2), st));
    } else {
        SIE_CUDA(pool_alloc(p, &s->d_band, size_t(ns) * std::max<int64_t>(s->nunk, 1) * (s->W + 1) * sizeof(double2), st));
        SIE_CUDA(pool_alloc(p, &s->d_bandc, size_t(ns) * std::max<int64_t>(s->nunk, 1) * (s->W + 1) * sizeof(double2), st));
    }
    const bool tiled = !s->nd && s->W <= 31 && s->nunk > 0;
    const bool wide = !s->nd && s->W > 31 && s->W < kWideMax && s->nunk > 0;
    const int64_t nband = int64_t(ns) * std::max<int64_t>(s->nunk, 1) * (s->W + 1);
    if (wide) {
        SIE_CUDA(pool_alloc(p, &s->d_band32, size_t(nband) * sizeof(float2), st));
        SIE_CUDA(pool_alloc(p, &s->d_bandc32, size_t(nband) * sizeof(float2), st));
    }
    const int64_t ntile = int64_t(ns) * 2 * s->nchunks * PC_TILE;
    if (tiled) {
        SIE_CUDA(pool_alloc(p, &s->d_tile64, size_t(ntile) * sizeof(double2), st));
        SIE_CUDA(pool_alloc(p, &s->d_tile32, size_t(ntile) * sizeof(float2), st));
        SIE_CUDA(pool_alloc(p, &s->d_dinv64, size_t(ns) * s->nunk * sizeof(double2), st));
        SIE_CUDA(pool_alloc(p, &s->d_dinv32, size_t(ns) * s->nunk * sizeof(float2), st));
        SIE_CUDA(pool_alloc(p, &s->d_tiledf, size_t(ntile) * sizeof(cdf), st));
        SIE_CUDA(pool_alloc(p, &s->d_dinvdf, size_t(ns) * s->nunk * sizeof(cdf), st));
        SIE_CUDA(pool_alloc(p, &s->d_adf, size_t(ns) * p->nb * sizeof(cdf), st));
    }
    SIE_CUDA(pool_alloc(p, &s->d_a, size_t(ns) * p->nb * sizeof(double2), st));
    SIE_CUDA(pool_alloc(p, &s->d_a32, size_t(ns) * p->nb * sizeof(float2), st));
    const int zw = 2 * p->ncond + 1;
    std::vector<double> zc(size_t(ns) * zw);
    for (int32_t f = 0; f < ns; ++f) {
        for (int c = 0; c < p->ncond; ++c) {
            const std::complex<double> z = surface_impedance(p, c, uniq[f]);
            zc[f * zw + 2 * c] = z.real();
            zc[f * zw + 2 * c + 1] = z.imag();
        }
        zc[f * zw + 2 * p->ncond] = uniq[f] * kMu0 / (4.0 * M_PI);
    }
    double *d_zc = nullptr;
    SIE_CUDA(pool_alloc(p, &d_zc, zc.size() * sizeof(double), st));
    SIE_CUDA(cudaMemcpyAsync(d_zc, zc.data(), zc.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    double2 *d_Lc = nullptr;   // lossy kernel: complex self terms per frequency slot
    if (p->params.kernel == SIE_KERNEL_LOSSY) {
        SIE_CUDA(pool_alloc(p, &d_Lc, size_t(ns) * std::max<int64_t>(p->nb, 1) * sizeof(double2), st));
        if (int rl = lossy_diag(p, uniq.data(), ns, d_Lc, st)) return rl;
    }
    k_pc_admittance<<<nblk_(p->nb * ns), 256, 0, st>>>(p->d_diag_gram, p->d_diag_L, d_Lc, p->d_br_cond, d_zc,
                                                       p->ncond, p->nb, ns, s->d_a);
    SIE_LAUNCH_CHECK(p);
    if (d_Lc) cudaFreeAsync(d_Lc, st);
    if (int rl = learned_admittance(p, d_zc, ns, s->d_a, st)) return rl;   // D' = D (1 + g)
    k_round_c<<<nblk_(p->nb * ns), 256, 0, st>>>(s->d_a, s->d_a32, p->nb * ns);
    SIE_LAUNCH_CHECK(p);
    if (tiled) {
        k_round_cdf<<<nblk_(p->nb * ns), 256, 0, st>>>(s->d_a, s->d_adf, p->nb * ns);
        SIE_LAUNCH_CHECK(p);
    }
    int zero = 0;
    SIE_CUDA(cudaMemcpyAsync(s->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    const int32_t nblk = int32_t(s->blk_off.size() - 1);
    StageTimer tm(p, SIE_STAGE_PRECOND_FACTOR, st);
    if (s->nd && s->nunk > 0) {
        // multifrontal LDL^T of each slot through one front workspace
        double2 *Wf = nullptr;
        SIE_CUDA(pool_alloc(p, &Wf, size_t(std::max<int64_t>(nd_workspace_size(s->nd), 1)) * sizeof(double2), st));
        const int64_t sl = nd_factor_size(s->nd);
        for (int32_t f = 0; f < ns; ++f) {
            const int rn = nd_factor(p, s->nd, s->d_a + int64_t(f) * p->nb, s->d_row_ptr, s->d_row_br, Wf,
                                     s->d_ndL64 + int64_t(f) * sl, s->d_ndL32 + int64_t(f) * sl, s->d_status, st);
            if (rn) {
                cudaFreeAsync(Wf, st);
                return rn;
            }
        }
        cudaFreeAsync(Wf, st);
    } else if (s->nunk > 0) {
        k_pc_factor<<<ns * nblk, 256, 0, st>>>(s->d_blk_off, nblk, s->W, s->nunk, s->d_row_ptr, s->d_row_br,
                                                s->d_row_oth, s->d_a, p->nb, s->d_band, s->d_bandc, s->d_status);
        SIE_LAUNCH_CHECK(p);
        if (tiled) {
            k_pc_tiles<double><<<nblk_(ntile), 256, 0, st>>>(s->d_band, s->d_bandc, s->d_blk_off, s->d_tile_off, nblk,
                                                               s->W, s->nunk, s->nchunks, ns, s->d_tile64);
            SIE_LAUNCH_CHECK(p);
            k_pc_tiles<float><<<nblk_(ntile), 256, 0, st>>>(s->d_band, s->d_bandc, s->d_blk_off, s->d_tile_off, nblk,
                                                              s->W, s->nunk, s->nchunks, ns, s->d_tile32);
            SIE_LAUNCH_CHECK(p);
            const int64_t nd = int64_t(ns) * s->nunk;
            k_pc_dinv<double><<<nblk_(nd), 256, 0, st>>>(s->d_band, nd, s->W + 1, s->d_dinv64);
            SIE_LAUNCH_CHECK(p);
            k_pc_dinv<float><<<nblk_(nd), 256, 0, st>>>(s->d_band, nd, s->W + 1, s->d_dinv32);
            SIE_LAUNCH_CHECK(p);
            k_pc_tiles<df><<<nblk_(ntile), 256, 0, st>>>(s->d_band, s->d_bandc, s->d_blk_off, s->d_tile_off, nblk,
                                                           s->W, s->nunk, s->nchunks, ns, s->d_tiledf);
            SIE_LAUNCH_CHECK(p);
            k_pc_dinv<df><<<nblk_(nd), 256, 0, st>>>(s->d_band, nd, s->W + 1, s->d_dinvdf);
            SIE_LAUNCH_CHECK(p);
        }
        if (wide) {
            k_round_c<<<nblk_(nband), 256, 0, st>>>(s->d_band, s->d_band32, nband);
            SIE_LAUNCH_CHECK(p);
            k_round_c<<<nblk_(nband), 256, 0, st>>>(s->d_bandc, s->d_bandc32, nband);
            SIE_LAUNCH_CHECK(p);
        }
    }
    int status = 0;
    SIE_CUDA(cudaMemcpyAsync(&status, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    cudaFreeAsync(d_zc, st);
    SIE_CUDA(cudaStreamSynchronize(st));
    if (status) return fail(SIE_ERR_BREAKDOWN, "preconditioner: zero pivot in the band LDL^T");
    s->slot_omega = uniq;
    s->nslots = ns;
    return SIE_OK;
}

// z = P^-1 y.  T = float: FP32 band factors and FP32 bookkeeping (mixed form,
// band width <= 31); T = double: everything in FP64.
template <typename T>
int pc_apply_t(pfft_plan *p, const double2 *y, double2 *z, int32_t R, cudaStream_t st) {
    PrecondState *s = p->pc;
    constexpr bool f32 = std::is_same<T, float>::value;
    constexpr bool dfl = std::is_same<T, df>::value;   // double-float: narrow bands only
    const int32_t nblk = int32_t(s->blk_off.size() - 1);
    C<T> *kappa = reinterpret_cast<C<T> *>(s->d_kappa);   // buffers sized for complex128
    C<T> *ibr = reinterpret_cast<C<T> *>(s->d_ibr);
    C<T> *u;
    const C<T> *a;
    if constexpr (f32) { u = s->d_u32; a = s->d_a32; }
    else if constexpr (dfl) { u = reinterpret_cast<cdf *>(s->d_u); a = s->d_adf; }
    else { u = s->d_u; a = s->d_a; }
    k_pc_drive<T><<<nblk_(p->nb * R), 256, 0, st>>>(y, p->nl, a, s->d_slot, p->d_loop_of_branch, p->d_tail,
                                                    p->d_head, s->d_off_ptr, s->d_off_port, s->d_off_sign,
                                                    s->d_port_loop, p->nb, R, kappa);
    SIE_LAUNCH_CHECK(p);
    if constexpr (dfl) {
        if (s->nd || s->W > 31 || !s->d_tiledf) return fail(SIE_ERR_ARG, "preconditioner: double-float sweeps "
                                                                         "need the narrow band route");
        if (s->nunk > 0) {
            k_pc_rhs<T><<<nblk_(int64_t(R) * s->nunk), 256, 0, st>>>(kappa, s->d_row_ptr, s->d_row_br, s->d_row_sg,
                                                                       s->nunk, p->nb, R, u);
            SIE_LAUNCH_CHECK(p);
            const size_t sm = size_t(4) * pc_nbuf<T>() * PC_TILE * sizeof(C<T>);
            if (int rc = set_smem((const void *)k_pc_sweep<T>, sm)) return rc;
            k_pc_sweep<T><<<nblk_(int64_t(R) * nblk * 32, 128), 128, sm, st>>>(
                s->d_blk_off, s->d_tile_off, nblk, s->nunk, s->nchunks, s->d_tiledf, s->d_dinvdf, s->d_slot, R, u);
            SIE_LAUNCH_CHECK(p);
        }
    } else if (s->nd && s->nunk > 0) {
        k_pc_rhs<T><<<nblk_(int64_t(R) * s->nunk), 256, 0, st>>>(kappa, s->d_row_ptr, s->d_row_br, s->d_row_sg,
                                                                   s->nunk, p->nb, R, u);
        SIE_LAUNCH_CHECK(p);
        const C<T> *Lf;
        if constexpr (f32) Lf = s->d_ndL32; else Lf = s->d_ndL64;
        int rn = nd_solve<T>(p, s->nd, Lf, s->d_slot, s->d_grp, s->ngrp, u, reinterpret_cast<C<T> *>(s->d_uv), st);
        if (rn) return rn;
    } else if (s->nunk > 0) {
        if (s->W <= 31) {
            k_pc_rhs<T><<<nblk_(int64_t(R) * s->nunk), 256, 0, st>>>(kappa, s->d_row_ptr, s->d_row_br, s->d_row_sg,
                                                                       s->nunk, p->nb, R, u);
            SIE_LAUNCH_CHECK(p);
            // four warps per CTA, pc_nbuf tiles of shared memory per warp
            const size_t sm = size_t(4) * pc_nbuf<T>() * PC_TILE * sizeof(C<T>);
            if (int rc = set_smem((const void *)k_pc_sweep<T>, sm)) return rc;
            const C<T> *tiles, *dinv;
            if constexpr (f32) { tiles = s->d_tile32; dinv = s->d_dinv32; } else { tiles = s->d_tile64; dinv = s->d_dinv64; }
            k_pc_sweep<T><<<nblk_(int64_t(R) * nblk * 32, 128), 128, sm, st>>>(
                s->d_blk_off, s->d_tile_off, nblk, s->nunk, s->nchunks, tiles, dinv, s->d_slot, R, u);
        } else if (s->W < kWideMax) {
            const int wt = (s->W + 1 + 31) / 32 * 32;
            const C<T> *band, *bandc;
            if constexpr (f32) { band = s->d_band32; bandc = s->d_bandc32; } else { band = s->d_band; bandc = s->d_bandc; }
            // blocked sweeps: Wt >= W threads, window of S >= W + 32 rows in shared memory
            int S = 64;
            while (S < s->W + 32) S *= 2;
            const size_t sm = size_t(S + 32 * 33 + 32) * sizeof(C<T>);
            if (wt <= 256) {
                if (int rc = set_smem((const void *)k_pc_sweep_blk<T, 256>, sm)) return rc;
                k_pc_sweep_blk<T, 256><<<unsigned(int64_t(R) * nblk), wt, sm, st>>>(
                    kappa, s->d_row_ptr, s->d_row_br, s->d_row_sg, s->d_blk_off, nblk, s->W, S, s->nunk, p->nb, band,
                    bandc, s->d_slot, u);
            } else {
                if (int rc = set_smem((const void *)k_pc_sweep_blk<T, 1024>, sm)) return rc;
                k_pc_sweep_blk<T, 1024><<<unsigned(int64_t(R) * nblk), wt, sm, st>>>(
                    kappa, s->d_row_ptr, s->d_row_br, s->d_row_sg, s->d_blk_off, nblk, s->W, S, s->nunk, p->nb, band,
                    bandc, s->d_slot, u);
            }
        } else {
            if constexpr (f32) return fail(SIE_ERR_ARG, "preconditioner: FP32 sweeps need a band width below 1024");
            else
                k_pc_solve<<<nblk_(int64_t(R) * nblk * 32, 128), 128, 0, st>>>(
                    kappa, s->d_row_ptr, s->d_row_br, s->d_row_sg, s->d_blk_off, nblk, s->W, s->nunk, p->nb,
                    s->d_band, s->d_slot, R, u);
        }
        SIE_LAUNCH_CHECK(p);
    }
    k_pc_currents<T><<<nblk_(p->nb * R), 256, 0, st>>>(u, s->nunk, kappa, a, s->d_slot, s->d_unk_of_node,
                                                       p->d_tail, p->d_head, p->nb, R, ibr);
    SIE_LAUNCH_CHECK(p);
    k_pc_out<T><<<nblk_(p->nl * R), 256, 0, st>>>(ibr, p->d_link_branch, s->d_src_ptr, s->d_src_br, s->d_src_sg,
                                                  p->nb, p->nl, R, z);
    SIE_LAUNCH_CHECK(p);
    return SIE_OK;
}

// Narrow band route (one warp per sweep): the one with double-float sweeps.
bool pc_df_route(const pfft_plan *p) { return p->pc && !p->pc->nd && p->pc->W <= 31 && p->pc->d_tiledf; }

int pc_apply_async(pfft_plan *p, const double2 *y, double2 *z, int32_t R, int prec, cudaStream_t st) {
    StageTimer tm(p, SIE_STAGE_PRECOND_APPLY, st);
    if (prec == SIE_PREC_MIXED && (p->pc->nd || p->pc->W < kWideMax)) return pc_apply_t<float>(p, y, z, R, st);
    if (prec == SIE_PREC_DF && pc_df_route(p)) return pc_apply_t<df>(p, y, z, R, st);
    return pc_apply_t<double>(p, y, z, R, st);   // FP64 (and double-float where no narrow band)
}

// ------------------------------------------------------------------ GMRES kernels

// Krylov basis layout [m+1][R][n]: vector j of right-hand side r at
// V + j * kstride + r * ldv, so each basis vector is a contiguous [R][n] block
// the batched matvec can take directly.
// h[r][j] = <V_j[r], w[r]> for j < k (one CTA per (r, j), k CTAs per right-hand
// side).  With kdev, only j <= *kdev are taken (the Arnoldi step index read on
// the device, so that one captured launch serves every step).
__global__ void k_dots(const double2 *__restrict__ V, int64_t ldv, int64_t kstride, const double2 *__restrict__ w,
                       int64_t n, int32_t k, const int32_t *__restrict__ active, double2 *__restrict__ h, int32_t ldh,
                       const int32_t *__restrict__ kdev = nullptr) {
    const int32_t r = blockIdx.x / k, j = blockIdx.x % k;
    if (!active[r]) return;
    if (kdev && j > *kdev) return;
    const double2 *v = V + int64_t(j) * kstride + int64_t(r) * ldv;
    const double2 *x = w + int64_t(r) * ldv;
    double re = 0.0, im = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double2 a = v[i], b = x[i];
        re += a.x * b.x + a.y * b.y;   // conj(a) b
        im += a.x * b.y - a.y * b.x;
    }
    __shared__ double sr[32], si[32];
    for (int s = 16; s > 0; s >>= 1) { re += __shfl_xor_sync(0xffffffffu, re, s); im += __shfl_xor_sync(0xffffffffu, im, s); }
    if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = re; si[threadIdx.x >> 5] = im; }
    __syncthreads();
    if (threadIdx.x < 32) {
        re = threadIdx.x < blockDim.x / 32 ? sr[threadIdx.x] : 0.0;
        im = threadIdx.x < blockDim.x / 32 ? si[threadIdx.x] : 0.0;
        for (int s = 16; s > 0; s >>= 1) { re += __shfl_xor_sync(0xffffffffu, re, s); im += __shfl_xor_sync(0xffffffffu, im, s); }
        if (threadIdx.x == 0) h[int64_t(r) * ldh + j] = make_double2(re, im);
    }
}

// w[r] -= sum_{j<k} h[r][j] V_j[r]   (k = *kdev + 1 with kdev)
__global__ void k_orth_update(const double2 *__restrict__ V, int64_t ldv, int64_t kstride, double2 *__restrict__ w,
                              int64_t n, int32_t k, const int32_t *__restrict__ active, const double2 *__restrict__ h,
                              int32_t ldh, int32_t R, const int32_t *__restrict__ kdev = nullptr) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n * R) return;
    int64_t r = i / n, e = i % n;
    if (!active[r]) return;
    if (kdev) k = *kdev + 1;
    double2 acc = w[r * ldv + e];
    const double2 *hr = h + r * ldh;
    const double2 *v = V + r * ldv + e;
    for (int32_t j = 0; j < k; ++j) acc = csub(acc, cmul(hr[j], v[int64_t(j) * kstride]));
    w[r * ldv + e] = acc;
}

// V_k[r] = w[r] * scale[r] (k = *kdev + 1 with kdev), also into vin when given
// (the fixed input buffer of the next step's product)
__global__ void k_scale_store(const double2 *__restrict__ w, int64_t ldv, double2 *__restrict__ V, int64_t kstride,
                              int32_t k, int64_t n, const double *__restrict__ scale, const int32_t *__restrict__ active,
                              int32_t R, const int32_t *__restrict__ kdev = nullptr, double2 *__restrict__ vin = nullptr) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n * R) return;
    int64_t r = i / n, e = i % n;
    if (!active[r]) return;
    if (kdev) k = *kdev + 1;
    const double2 v = cscale(w[r * ldv + e], scale[r]);
    V[int64_t(k) * kstride + r * ldv + e] = v;
    if (vin) vin[r * ldv + e] = v;
}

__global__ void k_step_advance(int32_t *kdev) { *kdev += 1; }

// x[r] += sum_j y[r][j] V_j[r]
__global__ void k_update_x(const double2 *__restrict__ V, int64_t ldv, int64_t kstride, double2 *__restrict__ x,
                           int64_t n, const int32_t *__restrict__ kr, const double2 *__restrict__ y, int32_t ldy,
                           int32_t R) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n * R) return;
    int64_t r = i / n, e = i % n;
    double2 acc = x[r * ldv + e];
    for (int32_t j = 0; j < kr[r]; ++j) acc = cadd(acc, cmul(y[r * ldy + j], V[int64_t(j) * kstride + r * ldv + e]));
    x[r * ldv + e] = acc;
}

__global__ void k_sub(const double2 *__restrict__ a, const double2 *__restrict__ b, double2 *__restrict__ c, int64_t n) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) c[i] = csub(a[i], b[i]);
}

__global__ void k_add(double2 *__restrict__ a, const double2 *__restrict__ b, int64_t n) {
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) a[i] = cadd(a[i], b[i]);
}

// Device state of one GMRES cycle per right-hand side r (Eq. LoopWithP):
// Hessenberg matrix after the rotations H[r][j][k] (pitch m), rotations
// cs[r][k], sn[r][k], rotated right-hand side g[r][0..m], steps taken kdone,
// total iterations iters, residual estimate resid = |g[k]| / bnorm, run flag.
struct GmresDev {
    double2 *H, *cs, *sn, *g;
    int32_t *run, *kdone, *iters;
    double *resid, *bnorm, *scale;
    int32_t *nrun, *bad;
};

// Start of a cycle: g = (beta, 0, ...), kdone = 0, scale = 1/beta for v_0,
// run = act (the right-hand sides still to converge).
__global__ void k_cycle_start(GmresDev d, int32_t m, int32_t R, const double *__restrict__ beta,
                              const int32_t *__restrict__ act) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    d.g[int64_t(r) * (m + 1)] = make_double2(beta[r], 0.0);
    d.kdone[r] = 0;
    d.run[r] = act[r];
    d.scale[r] = beta[r] > 0.0 ? 1.0 / beta[r] : 0.0;
}

// The end of Arnoldi step k per right-hand side (one thread each): column k of
// the Hessenberg matrix, h_jk = h1_j + h2_j (classical Gram-Schmidt applied
// twice) and h_{k+1,k} = ||w||; the previous rotations applied to it; the new
// rotation [[conj c, conj s], [-s, c]] that annihilates h_{k+1,k}; g rotated;
// the residual estimate |g_{k+1}| / bnorm; the scale 1/h_{k+1,k} of v_{k+1}.
// The run flag drops on convergence (resid < tol), on the iteration cap, on a
// happy breakdown (h_{k+1,k} = 0) or on a non-finite norm (bad is set); nrun
// counts the right-hand sides still running.
__global__ void k_givens(GmresDev d, int32_t k, int32_t m, int32_t R, const double2 *__restrict__ h1,
                         const double2 *__restrict__ h2, int32_t ldh, const double *__restrict__ hn, double tol,
                         int32_t max_iter, const int32_t *__restrict__ kdev = nullptr) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    if (kdev) k = *kdev;
    if (!d.run[r]) {
        d.scale[r] = 0.0;
        return;
    }
    const double hk1 = hn[r];
    if (!isfinite(hk1)) {
        d.run[r] = 0;
        d.scale[r] = 0.0;
        atomicExch(d.bad, 1);
        return;
    }
    double2 *Hc = d.H + int64_t(r) * (m + 1) * m;
    const double2 *cs = d.cs + int64_t(r) * m, *sn = d.sn + int64_t(r) * m;
    for (int32_t j = 0; j <= k; ++j) Hc[int64_t(j) * m + k] = cadd(h1[int64_t(r) * ldh + j], h2[int64_t(r) * ldh + j]);
    for (int32_t i = 0; i < k; ++i) {
        const double2 a = Hc[int64_t(i) * m + k], b = Hc[int64_t(i + 1) * m + k];
        const double2 c = cs[i], s = sn[i];
        // conj(c) a + conj(s) b and -s a + c b
        Hc[int64_t(i) * m + k] = make_double2(c.x * a.x + c.y * a.y + s.x * b.x + s.y * b.y,
                                              c.x * a.y - c.y * a.x + s.x * b.y - s.y * b.x);
        Hc[int64_t(i + 1) * m + k] = csub(cmul(c, b), cmul(s, a));
    }
    const double2 a = Hc[int64_t(k) * m + k];
    const double den = sqrt(a.x * a.x + a.y * a.y + hk1 * hk1);
    const double2 c = den > 0.0 ? make_double2(a.x / den, a.y / den) : make_double2(1.0, 0.0);
    const double2 s = den > 0.0 ? make_double2(hk1 / den, 0.0) : make_double2(0.0, 0.0);
    d.cs[int64_t(r) * m + k] = c;
    d.sn[int64_t(r) * m + k] = s;
    Hc[int64_t(k) * m + k] = make_double2(den, 0.0);
    double2 *g = d.g + int64_t(r) * (m + 1);
    const double2 gk = g[k];
    g[k + 1] = make_double2(-(s.x * gk.x - s.y * gk.y), -(s.x * gk.y + s.y * gk.x));
    g[k] = make_double2(c.x * gk.x + c.y * gk.y, c.x * gk.y - c.y * gk.x);
    d.kdone[r] = k + 1;
    d.iters[r] += 1;
    const double2 gn = g[k + 1];
    d.resid[r] = sqrt(gn.x * gn.x + gn.y * gn.y) / d.bnorm[r];
    d.scale[r] = hk1 > 0.0 ? 1.0 / hk1 : 0.0;
    if (d.resid[r] < tol || d.iters[r] >= max_iter || hk1 == 0.0) d.run[r] = 0;
    else atomicAdd(d.nrun, 1);
}

// y = R^-1 g of the cycle per right-hand side (back substitution in the rotated
// Hessenberg matrix), written to y[r][0..kdone).
__global__ void k_lsq(GmresDev d, int32_t m, int32_t R, double2 *__restrict__ y, int32_t ldy) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int32_t kk = d.kdone[r];
    const double2 *Hc = d.H + int64_t(r) * (m + 1) * m;
    const double2 *g = d.g + int64_t(r) * (m + 1);
    double2 *yr = y + int64_t(r) * ldy;
    for (int32_t i = kk - 1; i >= 0; --i) {
        double2 sum = g[i];
        for (int32_t j = i + 1; j < kk; ++j) sum = csub(sum, cmul(Hc[int64_t(i) * m + j], yr[j]));
        const double2 h = Hc[int64_t(i) * m + i];
        const double dd = h.x * h.x + h.y * h.y;
        yr[i] = make_double2((sum.x * h.x + sum.y * h.y) / dd, (sum.y * h.x - sum.x * h.y) / dd);
    }
}

// norms[r] = ||w[r]|| from the dot of w with itself (k_dots output h[r][0]).
__global__ void k_norms(const double2 *__restrict__ h, int32_t ldh, int32_t R, double *__restrict__ out) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) out[r] = sqrt(fmax(h[int64_t(r) * ldh].x, 0.0));
}

}  // namespace

extern "C" int pfft_precond_apply(pfft_plan *p, const void *y, void *z, int32_t nrhs, const double *omega,
                                  int32_t prec, void *cuda_stream) {
    if (!p || !y || !z || !omega || nrhs < 1) return fail(SIE_ERR_ARG, "pfft_precond_apply: bad argument");
    if (prec != SIE_PREC_FP64 && prec != SIE_PREC_MIXED && prec != SIE_PREC_DF)
        return fail(SIE_ERR_ARG, "pfft_precond_apply: bad precision");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    (void)cudaGetLastError();
    std::vector<int32_t> slot;
    int rc = pc_prepare(p, omega, nrhs, slot, st);
    if (rc) return rc;
    rc = pc_apply_async(p, (const double2 *)y, (double2 *)z, nrhs, prec, st);
    if (rc) return rc;
    SIE_CUDA(cudaStreamSynchronize(st));
    return SIE_OK;
}

namespace sie {

// One port solve (Eq. LoopWithP) as a sequence of steps, so that sie_solve can
// drive it eagerly and a batch can capture one Arnoldi step of many plans into
// one CUDA graph and replay it (the step reads its index k on the device and
// takes its product's input from the fixed buffer vin).
struct GmresRun {
    pfft_plan *p = nullptr;
    cudaStream_t st = nullptr;
    sie_solve_opts o{};
    int32_t nf = 0, np = 0, R = 0, m = 0;
    int64_t n = 0, ldv = 0, kstride = 0;
    std::vector<double> om;
    std::vector<int32_t> ports;
    bool use_pc = true, refine = false;
    int outer_prec = SIE_PREC_FP64;
    int resid_prec = SIE_PREC_FP64;   // the refinement's residual products: FP64 or double-float
    int pc_prec = SIE_PREC_FP64;      // the preconditioner inside the cycles
    int outer_pc_prec = SIE_PREC_FP64;   // the preconditioner of the convergence tests
    // device
    double2 *V = nullptr, *w = nullptr, *b = nullptr, *x = nullptr, *t = nullptr, *dh = nullptr, *dh2 = nullptr,
            *dhn = nullptr, *dy = nullptr, *rv = nullptr, *dvec = nullptr, *vin = nullptr;
    int32_t *act = nullptr, *kdev = nullptr;
    double *dnorm = nullptr, *dbeta = nullptr;
    GmresDev gd{};
    int32_t *hflags = nullptr;   // pinned: running right-hand sides, breakdown
    // host
    std::vector<int32_t> active, done, iters;
    std::vector<double> bnorm, resid;
    int64_t matvecs = 0;
    bool breakdown = false, first = true, mixed_since_fp64 = false;
    double cycle_start = 1.0, tol_inner = 0.0, rho_fp64 = 0.0;
    int32_t k_host = 0;
    std::chrono::steady_clock::time_point t0;

    ~GmresRun() {
        for (void *a : {(void *)V, (void *)w, (void *)b, (void *)x, (void *)t, (void *)dh, (void *)dh2, (void *)dhn,
                        (void *)dy, (void *)rv, (void *)dvec, (void *)vin, (void *)act, (void *)kdev, (void *)dnorm,
                        (void *)dbeta, (void *)gd.H, (void *)gd.cs, (void *)gd.sn, (void *)gd.g, (void *)gd.run,
                        (void *)gd.kdone, (void *)gd.iters, (void *)gd.resid, (void *)gd.bnorm, (void *)gd.scale,
                        (void *)gd.nrun})
            if (a) cudaFreeAsync(a, st);
        if (hflags) cudaFreeHost(hflags);
    }
    // out = P^-1 Z in (the product from the fixed coefficients; launch = true: no
    // coefficient upload, the form a graph captures)
    int apply_op(const double2 *in, double2 *out, int prec, bool launch_only) {
        int r2 = launch_only ? matvec_launch(p, in, use_pc ? t : out, R, SIE_SPACE_LOOP, prec, st)
                             : matvec_async(p, in, use_pc ? t : out, R, om.data(), SIE_SPACE_LOOP, prec, st);
        if (r2) return r2;
        if (use_pc) return pc_apply_async(p, t, out, R, prec == o.prec ? pc_prec : prec, st);
        return SIE_OK;
    }
    // ||vec[r]|| into dnorm (device) through k_dots on a one-vector basis
    int norms_dev(const double2 *vec, const int32_t *mask) {
        k_dots<<<R, 256, 0, st>>>(vec, ldv, ldv, vec, n, 1, mask, dhn, 1);
        SIE_LAUNCH_CHECK(p);
        k_norms<<<unsigned((R + 127) / 128), 128, 0, st>>>(dhn, 1, R, dnorm);
        SIE_LAUNCH_CHECK(p);
        return SIE_OK;
    }
    int read_norms(std::vector<double> &nr) {
        nr.resize(R);
        SIE_CUDA(cudaMemcpyAsync(nr.data(), dnorm, size_t(R) * sizeof(double), cudaMemcpyDeviceToHost, st));
        SIE_CUDA(cudaStreamSynchronize(st));
        return SIE_OK;
    }
    // residual r = b - Z x with the FP64-class product (FP64, or double-float on
    // the FP32 pipes with opts.refine = 2)
    int residual_fp64() {
        int rc = matvec_async(p, x, t, R, om.data(), SIE_SPACE_LOOP, resid_prec, st);
        if (rc) return rc;
        k_sub<<<nblk_(int64_t(R) * n), 256, 0, st>>>(b, t, rv, int64_t(R) * n);
        SIE_LAUNCH_CHECK(p);
        matvecs += R;
        return SIE_OK;
    }
};

int gmres_create(pfft_plan *p, const double *freqs, int32_t nf, const int32_t *ports, int32_t np,
                 const sie_solve_opts *opts, cudaStream_t st, GmresRun **out) {
    *out = nullptr;
    if (!p || !freqs || nf < 1 || !ports || np < 1 || !opts) return fail(SIE_ERR_ARG, "sie_solve: bad argument");
    for (int32_t i = 0; i < np; ++i)
        if (ports[i] < 0 || ports[i] >= p->np) return fail(SIE_ERR_ARG, "sie_solve: port index out of range");
    for (int32_t i = 0; i < nf; ++i)
        if (!(freqs[i] > 0.0 || (freqs[i] == 0.0 && dc_defined(p))) || !std::isfinite(freqs[i]))
            return fail(SIE_ERR_ARG, "sie_solve: frequencies must be positive (DC needs the slab surface model on "
                                     "every conductor: the classic surface impedance vanishes there)");
    if (!(opts->tol > 0.0) || opts->max_iter < 1) return fail(SIE_ERR_ARG, "sie_solve: bad tolerance or iteration cap");
    if (opts->prec != SIE_PREC_FP64 && opts->prec != SIE_PREC_MIXED) return fail(SIE_ERR_ARG, "sie_solve: bad precision");
    if (opts->refine < 0 || opts->refine > 2) return fail(SIE_ERR_ARG, "sie_solve: refine must be 0, 1 or 2");
    (void)cudaGetLastError();
    auto *g = new (std::nothrow) GmresRun;
    if (!g) return fail(SIE_ERR_OOM, "sie_solve: out of host memory");
    g->t0 = std::chrono::steady_clock::now();
    g->p = p;
    g->st = st;
    g->o = *opts;
    g->nf = nf;
    g->np = np;
    g->m = std::max(1, std::min(opts->restart, 1000));
    g->R = nf * np;
    g->n = p->nl;
    g->ldv = g->n;
    g->kstride = int64_t(g->R) * g->n;
    g->ports.assign(ports, ports + np);
    g->om.resize(g->R);
    for (int32_t f = 0; f < nf; ++f)
        for (int32_t q = 0; q < np; ++q) g->om[f * np + q] = 2.0 * M_PI * freqs[f];
    g->use_pc = opts->precond != 0;
    // iterative refinement: residuals and the convergence test in FP64
    g->outer_prec = (opts->refine && opts->prec == SIE_PREC_MIXED) ? SIE_PREC_FP64 : opts->prec;
    g->refine = g->outer_prec != opts->prec;
    if (g->refine && opts->refine == 2) {
        if (p->params.kernel != SIE_KERNEL_STATIC) {
            delete g;
            return fail(SIE_ERR_ARG, "sie_solve: double-float residuals (refine = 2) take the static kernel only");
        }
        g->resid_prec = SIE_PREC_DF;
    }
    g->rho_fp64 = 1e4 * opts->tol;
    auto bail = [&](int rc) { delete g; return rc; };
    const int32_t R = g->R, m = g->m;
    const int64_t n = g->n;
    std::vector<int32_t> slot;
    int rc;
    if (g->use_pc && (rc = pc_prepare(p, g->om.data(), R, slot, st))) return bail(rc);
    // the cycles' preconditioner: the product's precision, except that double-float
    // refinement (refine = 2) takes double-float sweeps where the band is narrow (the
    // FP32 sweeps of the nodal Laplacian's LDL^T limit how far one cycle can go)
    g->pc_prec = g->o.prec;
    if (g->refine && opts->refine == 2 && g->use_pc && pc_df_route(p)) g->pc_prec = SIE_PREC_DF;
    // the tests' P^-1 (b - Z x): FP64, or with refine = 2 on the narrow band route the
    // double-float sweeps (within 1e-11 of FP64, a third of its time)
    g->outer_pc_prec = g->pc_prec == SIE_PREC_DF ? SIE_PREC_DF : g->outer_prec;
#define GA(ptr, bytes) do { cudaError_t _e = pool_alloc(p, &(ptr), (bytes), st); if (_e != cudaSuccess) return bail(fail(_e == cudaErrorMemoryAllocation ? SIE_ERR_OOM : SIE_ERR_CUDA, std::string("sie_solve: workspace: ") + cudaGetErrorString(_e))); } while (0)
    GA(g->V, size_t(m + 1) * g->kstride * sizeof(double2));
    for (double2 **q : {&g->w, &g->b, &g->x, &g->t, &g->rv, &g->vin}) GA(*q, size_t(R) * n * sizeof(double2));
    if (g->refine) GA(g->dvec, size_t(R) * n * sizeof(double2));
    GA(g->dh, size_t(R) * (m + 2) * sizeof(double2));
    GA(g->dh2, size_t(R) * (m + 2) * sizeof(double2));
    GA(g->dhn, size_t(R) * sizeof(double2));
    GA(g->dy, size_t(R) * (m + 1) * sizeof(double2));
    GA(g->act, size_t(R) * sizeof(int32_t));
    GA(g->kdev, sizeof(int32_t));
    GA(g->dnorm, size_t(R) * sizeof(double));
    GA(g->dbeta, size_t(R) * sizeof(double));
    GA(g->gd.H, size_t(R) * (m + 1) * m * sizeof(double2));
    GA(g->gd.cs, size_t(R) * m * sizeof(double2));
    GA(g->gd.sn, size_t(R) * m * sizeof(double2));
    GA(g->gd.g, size_t(R) * (m + 1) * sizeof(double2));
    for (int32_t **q : {&g->gd.run, &g->gd.kdone, &g->gd.iters}) GA(*q, size_t(R) * sizeof(int32_t));
    for (double **q : {&g->gd.resid, &g->gd.bnorm, &g->gd.scale}) GA(*q, size_t(R) * sizeof(double));
    GA(g->gd.nrun, 2 * sizeof(int32_t));
#undef GA
    g->gd.bad = g->gd.nrun + 1;
    if (cudaMallocHost((void **)&g->hflags, 2 * sizeof(int32_t)) != cudaSuccess) {
        g->hflags = nullptr;
        return bail(fail(SIE_ERR_OOM, "sie_solve: pinned host allocation failed"));
    }
#define GC(call) do { cudaError_t _e = (call); if (_e != cudaSuccess) return bail(fail(SIE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e))); } while (0)
    GC(cudaMemsetAsync(g->V, 0, size_t(m + 1) * g->kstride * sizeof(double2), st));
    GC(cudaMemsetAsync(g->b, 0, size_t(R) * n * sizeof(double2), st));
    GC(cudaMemsetAsync(g->x, 0, size_t(R) * n * sizeof(double2), st));
    GC(cudaMemsetAsync(g->gd.iters, 0, size_t(R) * sizeof(int32_t), st));
    GC(cudaMemsetAsync(g->gd.nrun, 0, 2 * sizeof(int32_t), st));
    for (int32_t f = 0; f < nf; ++f)
        for (int32_t q = 0; q < np; ++q) {
            static const double2 one = make_double2(1.0, 0.0);
            int64_t pl = p->loops->loop_of_branch[p->nb + ports[q]];
            GC(cudaMemcpyAsync(g->b + int64_t(f * np + q) * n + pl, &one, sizeof(double2), cudaMemcpyHostToDevice, st));
        }
    g->active.assign(R, 1);
    g->done.assign(R, 0);
    g->iters.assign(R, 0);
    g->resid.assign(R, 1.0);
    GC(cudaMemcpyAsync(g->act, g->active.data(), R * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    // ||P^-1 b|| (the outer precision's preconditioner); r = b - Z x with x = 0
    if (g->use_pc) {
        if ((rc = pc_apply_async(p, g->b, g->w, R, g->outer_pc_prec, st))) return bail(rc);
    } else {
        GC(cudaMemcpyAsync(g->w, g->b, size_t(R) * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    }
    if ((rc = g->norms_dev(g->w, g->act))) return bail(rc);
    if ((rc = g->read_norms(g->bnorm))) return bail(rc);
    GC(cudaMemcpyAsync(g->gd.bnorm, g->dnorm, size_t(R) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    GC(cudaMemcpyAsync(g->rv, g->b, size_t(R) * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
#undef GC
    // the product's coefficients stay in the plan's scratch for the whole solve
    if ((rc = scratch_reserve(p, R, g->o.prec))) return bail(rc);
    if ((rc = scratch_reserve(p, R, g->outer_prec))) return bail(rc);
    if (g->resid_prec == SIE_PREC_DF && (rc = df_prepare(p, st))) return bail(rc);
    *out = g;
    return SIE_OK;
}

// Top of a cycle: the preconditioned residual and its norm (outer precision),
// convergence per right-hand side.  Iterative refinement: the cycles run the
// mixed operator on the current residual and x accumulates their corrections
// d; the mixed product's error scales with |Z| |x|, not |Z x|, so one cycle
// lowers the true residual by a bounded factor.  After a cycle the residual is
// updated as r = b - Z x with the FP64 product when the cycle started from a
// residual above 1e4 tol (relative to ||P^-1 b||), else as r = r - Z d with the
// mixed product (its error is relative to the small correction).  A
// convergence found on a residual that mixed updates produced is confirmed on
// the FP64 residual here, so the stopping test always rests on an FP64 product.
int gmres_top(GmresRun *g, bool &need) {
    pfft_plan *p = g->p;
    cudaStream_t st = g->st;
    const int32_t R = g->R;
    const int64_t n = g->n;
    need = false;
    for (;;) {
        int rc;
        if (g->use_pc) {
            if ((rc = pc_apply_async(p, g->rv, g->w, R, g->outer_pc_prec, st))) return rc;
        } else {
            SIE_CUDA(cudaMemcpyAsync(g->w, g->rv, size_t(R) * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        }
        if ((rc = g->norms_dev(g->w, g->act))) return rc;
        std::vector<double> beta;
        if ((rc = g->read_norms(beta))) return rc;
        bool any = false;
        g->cycle_start = 0.0;
        for (int32_t r = 0; r < R; ++r) {
            if (g->done[r] || !g->active[r]) {   // no new norm was taken for it
                g->active[r] = 0;
                continue;
            }
            g->resid[r] = g->bnorm[r] > 0 ? beta[r] / g->bnorm[r] : 0.0;
            if (!std::isfinite(g->resid[r])) g->breakdown = true;
            g->active[r] = !(g->resid[r] < g->o.tol) && g->iters[r] < g->o.max_iter && g->bnorm[r] > 0 &&
                           std::isfinite(g->resid[r]);
            if (g->resid[r] < g->o.tol) g->done[r] = 1;
            if (g->active[r]) g->cycle_start = std::max(g->cycle_start, g->resid[r]);
            any |= g->active[r] != 0;
        }
        if (!any && g->refine && g->mixed_since_fp64 && !g->breakdown) {
            if ((rc = g->residual_fp64())) return rc;
            g->mixed_since_fp64 = false;
            for (int32_t r = 0; r < R; ++r) {
                g->active[r] = g->iters[r] < g->o.max_iter && g->bnorm[r] > 0;
                g->done[r] = 0;
            }
            SIE_CUDA(cudaMemcpyAsync(g->act, g->active.data(), R * sizeof(int32_t), cudaMemcpyHostToDevice, st));
            continue;
        }
        need = any && !g->breakdown;
        return SIE_OK;
    }
}

int gmres_begin(GmresRun *g) {
    pfft_plan *p = g->p;
    cudaStream_t st = g->st;
    const int32_t R = g->R;
    SIE_CUDA(cudaMemcpyAsync(g->act, g->active.data(), R * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    SIE_CUDA(cudaMemcpyAsync(g->dbeta, g->dnorm, size_t(R) * sizeof(double), cudaMemcpyDeviceToDevice, st));
    SIE_CUDA(cudaMemcpyAsync(g->gd.iters, g->iters.data(), size_t(R) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    // the cycle's stopping level (relative to ||P^-1 b||): the tolerance, or with
    // refinement a fixed fraction of the largest starting residual, at least half the tolerance
    // (the reduction one cycle reaches on the bond-wire array: 1e-2 with the FP32
    // preconditioner, whose sweeps limit the cycle; 1e-3 with double-float sweeps,
    // measured against 1e-2 and 1e-4: 26 iterations against 32 and 28)
    const double per_cycle = g->pc_prec == SIE_PREC_DF ? 1e-3 : 1e-2;
    g->tol_inner = g->refine ? std::max(0.5 * g->o.tol, per_cycle * g->cycle_start) : g->o.tol;
    k_cycle_start<<<unsigned((R + 127) / 128), 128, 0, st>>>(g->gd, g->m, R, g->dbeta, g->act);
    SIE_LAUNCH_CHECK(p);
    k_scale_store<<<nblk_(int64_t(R) * g->n), 256, 0, st>>>(g->w, g->ldv, g->V, g->kstride, 0, g->n, g->gd.scale,
                                                             g->act, R, nullptr, g->vin);
    SIE_LAUNCH_CHECK(p);
    SIE_CUDA(cudaMemsetAsync(g->kdev, 0, sizeof(int32_t), st));
    g->k_host = 0;
    return SIE_OK;
}

// One Arnoldi step (CGS2) with the rotations on the device.  graph = true: every
// launch is independent of k (k read from kdev, dots over all m columns with the
// columns beyond k idle, the product from fixed coefficients), so that a
// captured step serves every step of the cycle.
int gmres_step(GmresRun *g, bool graph) {
    pfft_plan *p = g->p;
    cudaStream_t st = g->st;
    const int32_t R = g->R, m = g->m;
    const int64_t n = g->n;
    int rc = g->apply_op(g->vin, g->w, g->o.prec, graph);   // w = P^-1 Z v_k (counted in gmres_stepped)
    if (rc) return rc;
    StageTimer tm(p, SIE_STAGE_ARNOLDI, st);
    const int32_t K = graph ? m : g->k_host + 1;
    k_dots<<<R * K, 256, 0, st>>>(g->V, g->ldv, g->kstride, g->w, n, K, g->gd.run, g->dh, m + 2, g->kdev);
    SIE_LAUNCH_CHECK(p);
    k_orth_update<<<nblk_(int64_t(R) * n), 256, 0, st>>>(g->V, g->ldv, g->kstride, g->w, n, K, g->gd.run, g->dh,
                                                          m + 2, R, g->kdev);
    SIE_LAUNCH_CHECK(p);
    k_dots<<<R * K, 256, 0, st>>>(g->V, g->ldv, g->kstride, g->w, n, K, g->gd.run, g->dh2, m + 2, g->kdev);
    SIE_LAUNCH_CHECK(p);
    k_orth_update<<<nblk_(int64_t(R) * n), 256, 0, st>>>(g->V, g->ldv, g->kstride, g->w, n, K, g->gd.run, g->dh2,
                                                          m + 2, R, g->kdev);
    SIE_LAUNCH_CHECK(p);
    if ((rc = g->norms_dev(g->w, g->gd.run))) return rc;
    SIE_CUDA(cudaMemsetAsync(g->gd.nrun, 0, sizeof(int32_t), st));
    k_givens<<<unsigned((R + 127) / 128), 128, 0, st>>>(g->gd, 0, m, R, g->dh, g->dh2, m + 2, g->dnorm,
                                                         g->tol_inner, g->o.max_iter, g->kdev);
    SIE_LAUNCH_CHECK(p);
    k_scale_store<<<nblk_(int64_t(R) * n), 256, 0, st>>>(g->w, g->ldv, g->V, g->kstride, 0, n, g->gd.scale, g->gd.run,
                                                          R, g->kdev, g->vin);
    SIE_LAUNCH_CHECK(p);
    k_step_advance<<<1, 1, 0, st>>>(g->kdev);
    SIE_LAUNCH_CHECK(p);
    SIE_CUDA(cudaMemcpyAsync(g->hflags, g->gd.nrun, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    return SIE_OK;
}

// After the step's stream has synchronised: true when the cycle is over.
bool gmres_stepped(GmresRun *g) {
    g->k_host += 1;
    g->matvecs += g->R;
    if (g->hflags[1]) g->breakdown = true;
    return g->hflags[0] == 0 || g->k_host >= g->m || g->breakdown;
}

// End of a cycle: x += V y (y from the rotated Hessenberg matrix), convergence
// without refinement, the new residual.  cont = false: the solve is over.
int gmres_end(GmresRun *g, bool &cont) {
    pfft_plan *p = g->p;
    cudaStream_t st = g->st;
    const int32_t R = g->R, m = g->m;
    const int64_t n = g->n;
    cont = false;
    k_lsq<<<unsigned((R + 127) / 128), 128, 0, st>>>(g->gd, m, R, g->dy, m + 1);
    SIE_LAUNCH_CHECK(p);
    double2 *xd = g->refine ? g->dvec : g->x;
    if (g->refine) SIE_CUDA(cudaMemsetAsync(g->dvec, 0, size_t(R) * n * sizeof(double2), st));
    k_update_x<<<nblk_(int64_t(R) * n), 256, 0, st>>>(g->V, g->ldv, g->kstride, xd, n, g->gd.kdone, g->dy, m + 1, R);
    SIE_LAUNCH_CHECK(p);
    std::vector<double> rs(R);
    SIE_CUDA(cudaMemcpyAsync(g->iters.data(), g->gd.iters, size_t(R) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SIE_CUDA(cudaMemcpyAsync(rs.data(), g->gd.resid, size_t(R) * sizeof(double), cudaMemcpyDeviceToHost, st));
    SIE_CUDA(cudaStreamSynchronize(st));
    if (g->breakdown) return SIE_OK;
    // without refinement the cycle's residual estimate decides; with it the
    // residual at the top of the next cycle does
    if (!g->refine)
        for (int32_t r = 0; r < R; ++r)
            if (g->active[r]) {
                g->resid[r] = rs[r];
                if (rs[r] < g->o.tol) g->done[r] = 1;
            }
    bool more = false;
    for (int32_t r = 0; r < R; ++r) more |= !g->done[r] && g->iters[r] < g->o.max_iter;
    if (!more && !g->refine) return SIE_OK;
    for (int32_t r = 0; r < R; ++r) g->active[r] = !g->done[r] && g->iters[r] < g->o.max_iter;
    SIE_CUDA(cudaMemcpyAsync(g->act, g->active.data(), R * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    int rc;
    if (!g->refine) {
        if ((rc = matvec_async(p, g->x, g->t, R, g->om.data(), SIE_SPACE_LOOP, g->o.prec, st))) return rc;
        g->matvecs += R;
        k_sub<<<nblk_(int64_t(R) * n), 256, 0, st>>>(g->b, g->t, g->rv, int64_t(R) * n);
        SIE_LAUNCH_CHECK(p);
    } else {
        k_add<<<nblk_(int64_t(R) * n), 256, 0, st>>>(g->x, g->dvec, int64_t(R) * n);
        SIE_LAUNCH_CHECK(p);
        if (g->first || g->cycle_start > g->rho_fp64) {
            if ((rc = g->residual_fp64())) return rc;
            g->mixed_since_fp64 = false;
        } else {
            if ((rc = matvec_async(p, g->dvec, g->t, R, g->om.data(), SIE_SPACE_LOOP, g->o.prec, st))) return rc;
            k_sub<<<nblk_(int64_t(R) * n), 256, 0, st>>>(g->rv, g->t, g->rv, int64_t(R) * n);
            SIE_LAUNCH_CHECK(p);
            g->matvecs += R;
            g->mixed_since_fp64 = true;
        }
        g->first = false;
    }
    if (!more) {   // refinement: iteration cap reached; report the residual of the final x
        if (g->mixed_since_fp64 && (rc = g->residual_fp64())) return rc;
        if (g->use_pc) {
            if ((rc = pc_apply_async(p, g->rv, g->w, R, g->outer_pc_prec, st))) return rc;
        } else {
            SIE_CUDA(cudaMemcpyAsync(g->w, g->rv, size_t(R) * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        }
        if ((rc = g->norms_dev(g->w, g->act))) return rc;
        std::vector<double> fin;
        if ((rc = g->read_norms(fin))) return rc;
        for (int32_t r = 0; r < R; ++r)
            if (!g->done[r] && g->bnorm[r] > 0) g->resid[r] = fin[r] / g->bnorm[r];
        return SIE_OK;
    }
    cont = true;
    return SIE_OK;
}

// Port currents -> Y -> Z = Y^-1 per frequency, the statistics; frees the run.
int gmres_finish(GmresRun *g, sie_c64 *Z_out, sie_solve_stats *st_out) {
    using cd = std::complex<double>;
    pfft_plan *p = g->p;
    const int32_t R = g->R, nf = g->nf, np = g->np;
    const int64_t n = g->n;
    std::vector<double2> xh(size_t(R) * n);
    cudaError_t e = cudaMemcpyAsync(xh.data(), g->x, xh.size() * sizeof(double2), cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) {
        delete g;
        return fail(SIE_ERR_CUDA, std::string("sie_solve: ") + cudaGetErrorString(e));
    }
    int32_t nnc = 0, itmax = 0, itsum = 0;
    double rmax = 0.0;
    for (int32_t r = 0; r < R; ++r) {
        nnc += !(g->resid[r] < g->o.tol);
        itmax = std::max(itmax, g->iters[r]);
        itsum += g->iters[r];
        rmax = std::max(rmax, g->resid[r]);
    }
    int rc = SIE_OK;
    for (int32_t f = 0; f < nf && !rc; ++f) {
        // Y[q][p] = current in port q's loop with port p driven; Z = Y^-1 (Gauss-Jordan)
        std::vector<cd> Y(size_t(np) * np), Zi(size_t(np) * np, 0.0);
        for (int32_t q = 0; q < np; ++q)
            for (int32_t pp = 0; pp < np; ++pp) {
                int64_t pl = p->loops->loop_of_branch[p->nb + g->ports[q]];
                double2 v = xh[size_t(f * np + pp) * n + pl];
                Y[size_t(q) * np + pp] = cd(v.x, v.y);
            }
        for (int32_t i = 0; i < np; ++i) Zi[size_t(i) * np + i] = 1.0;
        for (int32_t c = 0; c < np && !rc; ++c) {
            int32_t piv = c;
            for (int32_t r2 = c + 1; r2 < np; ++r2)
                if (std::abs(Y[size_t(r2) * np + c]) > std::abs(Y[size_t(piv) * np + c])) piv = r2;
            for (int32_t j = 0; j < np; ++j) {
                std::swap(Y[size_t(c) * np + j], Y[size_t(piv) * np + j]);
                std::swap(Zi[size_t(c) * np + j], Zi[size_t(piv) * np + j]);
            }
            cd d = Y[size_t(c) * np + c];
            if (d == cd(0.0)) {
                rc = fail(SIE_ERR_BREAKDOWN, "sie_solve: singular port admittance matrix");
                break;
            }
            for (int32_t j = 0; j < np; ++j) { Y[size_t(c) * np + j] /= d; Zi[size_t(c) * np + j] /= d; }
            for (int32_t r2 = 0; r2 < np; ++r2) {
                if (r2 == c) continue;
                cd fct = Y[size_t(r2) * np + c];
                for (int32_t j = 0; j < np; ++j) {
                    Y[size_t(r2) * np + j] -= fct * Y[size_t(c) * np + j];
                    Zi[size_t(r2) * np + j] -= fct * Zi[size_t(c) * np + j];
                }
            }
        }
        for (int32_t i = 0; i < np * np && !rc; ++i) Z_out[size_t(f) * np * np + i] = sie_c64{Zi[i].real(), Zi[i].imag()};
    }
    if (st_out) {
        st_out->iterations_max = itmax;
        st_out->iterations_sum = itsum;
        st_out->n_not_converged = nnc;
        st_out->residual_max = rmax;
        st_out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - g->t0).count();
        st_out->matvecs = g->matvecs;
    }
    const bool breakdown = g->breakdown;
    delete g;
    if (rc) return rc;
    if (int dev_rc = check_device_errors(p)) return dev_rc;
    if (breakdown) return fail(SIE_ERR_BREAKDOWN, "sie_solve: non-finite value in the Arnoldi recurrence");
    if (nnc) return fail(SIE_ERR_NOT_CONVERGED, "sie_solve: " + std::to_string(nnc) + " right-hand sides did not converge");
    return SIE_OK;
}

void gmres_free(GmresRun *g) { delete g; }
cudaStream_t gmres_stream(const GmresRun *g) { return g->st; }
int64_t gmres_plan_launches(const GmresRun *g) { return g->p->launches; }

}  // namespace sie

extern "C" int sie_solve(pfft_plan *p, const double *freqs, int32_t nf, const int32_t *ports, int32_t np,
                         const sie_solve_opts *opts, sie_c64 *Z_out, sie_solve_stats *st_out) {
    if (!p || !Z_out) return fail(SIE_ERR_ARG, "sie_solve: bad argument");
    GmresRun *g = nullptr;
    int rc = gmres_create(p, freqs, nf, ports, np, opts, p->stream, &g);
    if (rc) return rc;
    for (;;) {
        bool need = false;
        if ((rc = gmres_top(g, need)) || !need) break;
        if ((rc = gmres_begin(g))) break;
        for (;;) {
            if ((rc = gmres_step(g, false))) break;
            if (cudaStreamSynchronize(g->st) != cudaSuccess) {
                rc = fail(SIE_ERR_CUDA, "sie_solve: Arnoldi step failed");
                break;
            }
            if (gmres_stepped(g)) break;
        }
        if (rc) break;
        bool cont = false;
        if ((rc = gmres_end(g, cont)) || !cont) break;
    }
    if (rc) {
        gmres_free(g);
        return rc;
    }
    return gmres_finish(g, Z_out, st_out);
}

// ------------------------------------------------------------------ surface model

namespace sie {
void invalidate_precond_factors(pfft_plan *p) {
    if (p->pc) p->pc->slot_omega.clear();
}
}  // namespace sie

extern "C" int pfft_precond_set_method(pfft_plan *p, int32_t method) {
    if (!p) return fail(SIE_ERR_ARG, "pfft_precond_set_method: NULL plan");
    if (method != SIE_PC_AUTO && method != SIE_PC_BAND && method != SIE_PC_ND)
        return fail(SIE_ERR_ARG, "pfft_precond_set_method: unknown method");
    if (method != p->pc_method) {
        cudaDeviceSynchronize();   // no solve of this plan may still use the state
        plan_free_precond(p);
        p->pc_method = method;
    }
    return SIE_OK;
}

extern "C" int pfft_precond_nd_info(pfft_plan *p, int32_t *method_used, int32_t *fronts, int64_t *nnz_factor,
                                    int32_t *max_front, int64_t *flops) {
    if (!p) return fail(SIE_ERR_ARG, "pfft_precond_nd_info: NULL plan");
    if (!p->pc) {
        int rc = build_symbolic(p);
        if (rc) { plan_free_precond(p); return rc; }
    }
    if (method_used) *method_used = p->pc->nd ? SIE_PC_ND : SIE_PC_BAND;
    if (fronts) *fronts = 0;
    if (nnz_factor) *nnz_factor = 0;
    if (max_front) *max_front = 0;
    if (flops) *flops = 0;
    if (p->pc->nd) nd_info(p->pc->nd, fronts, nnz_factor, max_front, flops);
    return SIE_OK;
}

extern "C" int pfft_precond_info(pfft_plan *p, int32_t *band_width, int64_t *unknowns, int64_t *blocks) {
    if (!p) return fail(SIE_ERR_ARG, "pfft_precond_info: NULL plan");
    if (!p->pc) {
        int rc = build_symbolic(p);
        if (rc) { plan_free_precond(p); return rc; }
    }
    if (band_width) *band_width = p->pc->W;
    if (unknowns) *unknowns = p->pc->nunk;
    if (blocks) *blocks = int64_t(p->pc->blk_off.size()) - 1;
    return SIE_OK;
}

extern "C" int pfft_plan_set_surface_model(pfft_plan *p, const double *t_eff, int32_t ncond) {
    if (!p) return fail(SIE_ERR_ARG, "pfft_plan_set_surface_model: NULL plan");
    if (ncond != p->ncond)
        return fail(SIE_ERR_ARG, "pfft_plan_set_surface_model: ncond must equal the mesh's conductor count (" +
                                     std::to_string(p->ncond) + ")");
    std::vector<double> t(size_t(ncond), 0.0);
    if (t_eff)
        for (int32_t c = 0; c < ncond; ++c) {
            if (!(t_eff[c] >= 0.0) || !std::isfinite(t_eff[c]))
                return fail(SIE_ERR_ARG, "pfft_plan_set_surface_model: thickness must be finite and >= 0");
            t[c] = t_eff[c];
        }
    p->t_eff = t;
    if (p->pc) p->pc->slot_omega.clear();   // the cached factors were built with the previous Z_s
    return SIE_OK;
}
