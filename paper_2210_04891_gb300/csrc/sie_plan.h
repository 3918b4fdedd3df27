// pFFT plan: everything the matvec, the preconditioner and the solver need,
// resident in device memory for the plan's lifetime.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <complex>
#include <vector>

#include "sie_common.cuh"

namespace sie {

template <typename T> struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
};

// Projection chunks of the mixed form (k_project_tiled): at most kChunkTri
// triangles staged per chunk, kChunkRhs right-hand sides per slab.
constexpr int kChunkTri = 64;
constexpr int kChunkRhs = 32;

struct PrecondState;   // sie_solve.cu
struct LossyCache;     // sie_lossy.cu
struct NdState;        // sie_nd.cu

struct Scratch {
    int32_t cap_rhs = 0;   // right-hand sides the buffers are sized for
    int cs = 0;            // complex element size the buffers are sized for (8 or 16)
    // tour, y_tri and y_br hold complex128 in the FP64 form and double-float
    // complex (float4: re hi, re lo, im hi, im lo) in the mixed form
    void *tour = nullptr;      // [R][2 n_nodes]
    void *grid = nullptr;      // complex T [3][R][Ng]   grid currents, then grid potentials
    void *spec = nullptr;      // complex T [3R][Mx][Ny][Nz]  grids transformed along x, then (large
                               // planes) [3R][Mx][My][Nz] the same transformed along y
    void *phiT = nullptr;      // complex T [Ng][3][R]   grid potentials, right-hand sides innermost
    void *y_tri = nullptr;     // [R][nt][3]
    void *y_br = nullptr;      // [R][nb + np]
    // per RHS: Z_s per conductor (re, im), c_L (im) -> double [R][2 ncond + 1],
    // followed by the same table as double-float (hi, lo) pairs, see coef_dd()
    double *coef = nullptr;
    void *cT = nullptr;        // complex T [nt][3][R]  local currents, right-hand sides innermost
    void *ffar = nullptr;      // complex64 [nt][3][R]  interpolated far field (mixed form)
    size_t bytes = 0;
};

}  // namespace sie

struct pfft_plan {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t launches = 0;
    // sizes
    int64_t nt = 0, nb = 0, nl = 0, np = 0, nn = 0;
    int32_t ncond = 0;
    int Nx = 0, Ny = 0, Nz = 0, Mx = 0, My = 0, Mz = 0, O = 3, Q = 7;
    // the padded (y, z) plane does not fit one CTA: y pencils and z rows through device memory
    bool large_plane = false;
    // incremented whenever the scratch buffers are reallocated (captured graphs hold their addresses)
    uint64_t scr_gen = 0;
    // learned correction of the preconditioner's branch diagonal (borrowed; NULL: plain)
    const sie_mlp *learned = nullptr;
    // stream-ordered allocations of the solve path (GMRES workspaces, per-frequency factors):
    // the plan's own pool, which keeps freed memory mapped until the plan is destroyed
    cudaMemPool_t pool = nullptr;
    int64_t Ng = 0;
    double lo[3] = {0, 0, 0}, h[3] = {0, 0, 0};
    double r_near = 0.0;
    pfft_params params{};
    const sie_loops *loops = nullptr;   // borrowed: must outlive the plan
    std::vector<double> sigma;          // per conductor
    std::vector<double> tri_cen;        // [nt][3] triangle centroids (host; the preconditioner's
                                        // nested-dissection ordering bisects by position)
    int32_t pc_method = 0;              // SIE_PC_AUTO, SIE_PC_BAND or SIE_PC_ND
    sie_kernel_tuning kt{};             // kernel launch shapes (pfft_plan_set_kernel_tuning)
    std::vector<double> t_eff;          // per conductor: slab surface impedance thickness (0: classic)
    // per triangle (device)
    int32_t *d_tb = nullptr;            // [nt][3] branch of local edge k (-1: none)
    int8_t *d_ts = nullptr;             // [nt][3] +1 on T+, -1 on T-
    int32_t *d_cond = nullptr;          // [nt]
    double *d_gram = nullptr;           // [nt][3][3]  int (r-v_k).(r-v_l) dS / (4A^2)
    double *d_mom64 = nullptr;          // [nt*Q][3][3] (w_q/2)(r_q - v_k)
    float *d_mom32 = nullptr;
    int32_t *d_start = nullptr;         // [nt*Q][3] stencil start nodes
    double *d_lw64 = nullptr;           // [nt*Q][3][O] Lagrange weights
    float *d_lw32 = nullptr;
    // projection blocks, one per (grid node n, triangle T) pair:
    //   W(n, T)[d][k] = sum_q L_n(r_q) (w_q/2)(r_q - v_k)_d
    // stored twice as packed records (sie_common.cuh, Rec<T>)
    int64_t n_pair = 0;
    int64_t *d_pn_ptr = nullptr;        // [Ng + 1]  rows = nodes, triangles ascending
    sie::Rec<double> *d_pn_rec64 = nullptr;  //   b[3d + k] = W[d][k], col = T
    sie::Rec<float> *d_pn_rec32 = nullptr;
    int64_t *d_pt_ptr = nullptr;        // [nt + 1]  rows = triangles, nodes ascending
    sie::Rec<double> *d_pt_rec64 = nullptr;  //   b[3k + d] = W[d][k], col = n
    sie::Rec<float> *d_pt_rec32 = nullptr;
    // projection chunks of the mixed form (k_project_tiled): node tiles of
    // 2 x 4 x 8 (x, y, z) nodes, split where their triangles exceed kChunkTri;
    // a chunk's triangles are staged once per slab in shared memory and each
    // node record names its triangle by its index in the chunk (pn_lcol)
    int64_t n_pchunk = 0;
    int32_t *d_pch_node_ptr = nullptr;  // [n_pchunk + 1] into d_pch_nodes
    int32_t *d_pch_nodes = nullptr;     // nodes of each chunk, ascending
    int32_t *d_pch_tri_ptr = nullptr;   // [n_pchunk + 1] into d_pch_tri
    int32_t *d_pch_tri = nullptr;       // triangles of each chunk
    uint16_t *d_pn_lcol = nullptr;      // [n_pair] per node record: index of its triangle in the chunk
    int64_t n_tiles = 0;                // 32-node tiles that hold at least one stencil node
    int32_t *d_tiles = nullptr;         // [n_tiles] tile index n / 32, ascending
    // near field CSR over triangles (row T: near T', ascending), 3x3 blocks
    int64_t n_near = 0;
    int64_t *d_near_ptr = nullptr;
    int32_t *d_near_col = nullptr;
    double *d_Ld64 = nullptr;           // [n_near][3][3]  L_direct - L_grid
    double *d_Ldir64 = nullptr;         // [n_near][3][3]  L_direct (kept for diag and checks)
    sie::Rec<double> *d_near_rec64 = nullptr;   // [n_near] {b = L_d block [k][l], col = T'}
    sie::Rec<float> *d_near_rec32 = nullptr;
    // tensor-core near field: row tiles of 42 triangles, their column unions
    int64_t nm_tiles = 0, nm_union = 0;
    int64_t *d_nm_uptr = nullptr;       // [nm_tiles + 1] union offsets (even counts)
    int32_t *d_nm_utri = nullptr;       // [nm_union] column triangles, ascending per tile
    float *d_nm_A = nullptr;            // [nm_union][128][3] dense L_d blocks of each tile (fp32)
    int *d_err = nullptr;               // device error flags (a bounded wait ran out)
    int *h_err = nullptr;               // pinned host copy, read with the call's own stream sync
    // kernel spectrum, folded [My/2+1][Mz/2+1][Mx/2+1], scaled by 1/(Mx My Mz)
    double *d_H64 = nullptr;
    float *d_H32 = nullptr;
    double2 *d_tw64[3] = {nullptr, nullptr, nullptr};   // per axis, length M_d
    float2 *d_tw32[3] = {nullptr, nullptr, nullptr};
    // four-step twiddle tables per axis: tf[j2][k1] = W^(j2 k1), ti[k1][p2] = W^(k1 p2)
    double2 *d_tf64[3] = {nullptr, nullptr, nullptr}, *d_ti64[3] = {nullptr, nullptr, nullptr};
    float2 *d_tf32[3] = {nullptr, nullptr, nullptr}, *d_ti32[3] = {nullptr, nullptr, nullptr};
    // the same spectrum with kx outermost: [Mx/2+1][My/2+1][Mz/2+1]
    double *d_Hp64 = nullptr;
    float *d_Hp32 = nullptr;
    // double-float copies for the SIE_PREC_DF product, built on its first use
    // (df_prepare): block records, four-step twiddles, kernel spectrum
    bool df_ready = false;
    sie::Rec<sie::df> *d_pn_recdf = nullptr, *d_pt_recdf = nullptr, *d_near_recdf = nullptr;
    sie::cdf *d_tfdf[3] = {nullptr, nullptr, nullptr}, *d_tidf[3] = {nullptr, nullptr, nullptr};
    sie::df *d_Hpdf = nullptr;
    // lossy kernel exp(-jkR)/R: complex spectrum of the last (omega, sigma), same layout
    // (pfft_convolve_lossy)
    double lossy_omega = -1.0, lossy_sigma = -1.0;
    double2 *d_Hl64 = nullptr;
    float2 *d_Hl32 = nullptr;
    // the lossy kernel inside pfft_matvec (params.kernel == SIE_KERNEL_LOSSY): per-frequency
    // spectra, near blocks and branch diagonals (sie_lossy.cu), and the geometry their
    // set-up needs, kept on the device for the plan's lifetime
    sie::LossyCache *lossy = nullptr;
    double *d_verts = nullptr;          // [nt][3][3] vertices
    double *d_r7b = nullptr, *d_r7w = nullptr;   // Radon 7-point rule (barycentric [7][3], weights [7])
    // loop basis on the device
    int32_t *d_tour_node = nullptr;     // [2 nn]
    int8_t *d_tour_enter = nullptr;     // [2 nn]
    int32_t *d_enter = nullptr, *d_exit = nullptr;   // [nn]
    int32_t *d_nl_ptr = nullptr, *d_nl_loop = nullptr;
    int8_t *d_nl_sign = nullptr;
    int32_t *d_parent_branch = nullptr;  // [nn]
    int32_t *d_twig_node = nullptr;      // [nb]: node whose parent branch it is, -1 for links
    // post-processing: tour slot of each panel's node and of its conductor's reference node
    int32_t *d_panel_slot = nullptr, *d_panel_ref = nullptr;   // [nt]
    int32_t *d_loop_of_branch = nullptr; // [nb + np]
    int32_t *d_tail = nullptr, *d_head = nullptr;  // [nb + np]
    int32_t *d_link_branch = nullptr;    // [nl]
    int32_t *d_br_tri = nullptr;         // [nb][2]
    int8_t *d_br_local = nullptr;        // [nb][2]
    // branch diagonal of Z_b pieces (preconditioner, Eq. Precond)
    double *d_diag_gram = nullptr;       // [nb]
    double *d_diag_L = nullptr;          // [nb]
    int32_t *d_br_cond = nullptr;        // [nb]
    // stage timing
    bool prof_on = false;
    struct ProfEv { int stage; cudaEvent_t a, b; };
    std::vector<ProfEv> prof_pending;
    double prof_ms[SIE_NSTAGES] = {0};
    int64_t prof_count[SIE_NSTAGES] = {0};
    sie::Scratch scr;
    sie::PrecondState *pc = nullptr;
    size_t device_bytes = 0;
    std::vector<void *> allocations;
};

namespace sie {
// Brackets one stage with CUDA events on its stream when profiling is on.
struct StageTimer {
    pfft_plan *p;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    StageTimer(pfft_plan *plan, int st, cudaStream_t stream) : p(plan), stage(st), s(stream) {
        if (p->prof_on && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, s);
    }
    ~StageTimer() {
        if (!a) return;
        cudaEvent_t b;
        if (cudaEventCreate(&b) == cudaSuccess) {
            cudaEventRecord(b, s);
            p->prof_pending.push_back({stage, a, b});
        } else {
            cudaEventDestroy(a);
        }
    }
};
int plan_alloc(pfft_plan *p, void **ptr, size_t bytes);
// raise a kernel's dynamic shared-memory limit to at least bytes (thread-safe, never lowers it)
int set_smem(const void *fn, size_t bytes);
void plan_free(pfft_plan *p, void *ptr);
void plan_free_precond(pfft_plan *p);
int scratch_reserve(pfft_plan *p, int32_t nrhs, int prec);
// Builds the double-float tables of the SIE_PREC_DF product from the FP64 ones
// on stream st (once per plan; no-op afterwards).
int df_prepare(pfft_plan *p, cudaStream_t st);
// Surface impedance of conductor c at angular frequency w (Eq. ImpedanceOp):
// classic (1 + j) sqrt(w mu0 / (2 sigma)), or with an effective thickness
// t > 0 the impedance of one face of a slab of thickness t,
// (gamma / sigma) coth(gamma t / 2) with gamma = (1 + j) sqrt(w mu0 sigma / 2).
std::complex<double> surface_impedance(const pfft_plan *p, int c, double w);
float2 *coef_dd(const pfft_plan *p);   // double-float copy of scr.coef
// Per-right-hand-side scalars of Eq. Zb for omega[R] into host arrays cf[R (2 ncond + 1)]
// (FP64) and cd (the same as double-float pairs); SIE_ERR_ARG for a bad omega.
int fill_coef(const pfft_plan *p, const double *omega, int32_t R, double *cf, float2 *cd);
// The matvec's kernels on stream st, with scratch reserved and the coefficients
// of this batch already in scr.coef (matvec_async = reserve + upload + launch).
int matvec_launch(pfft_plan *p, const void *x, void *y, int32_t nrhs, int space, int prec, cudaStream_t st);
int matvec_async(pfft_plan *p, const void *x, void *y, int32_t nrhs, const double *omega, int space, int prec,
                 cudaStream_t st);
// Admittances a [nslots][nb] of the preconditioner scaled by 1 / (1 + g) when the plan
// has a learned network (no-op otherwise); d_zs_cl as in the preconditioner's set-up.
int learned_admittance(pfft_plan *p, const double *d_zs_cl, int32_t nslots, double2 *a, cudaStream_t st);
// Forget the preconditioner's cached numeric factors (rebuilt on next use).
void invalidate_precond_factors(pfft_plan *p);
template <typename T> const C<T> *twiddle(const pfft_plan *p, int axis);
// Kernel spectra chosen per grid (the lossy kernel of pfft_matvec): grid g of a
// convolution uses the folded complex spectrum tab[gslot[g]] (device arrays;
// tab holds double2 or float2 pointers for the FP64 and mixed forms).
struct SpecSel {
    const void *const *tab = nullptr;
    const int32_t *gslot = nullptr;
};
int fft_conv(pfft_plan *p, void *grid, void *spec, int32_t nrhs, int prec, cudaStream_t s,
             const SpecSel *sel = nullptr);
int fft_conv_n(pfft_plan *p, void *grid, void *spec, int32_t ngrids, int prec, cudaStream_t s,
               bool lossy = false, const SpecSel *sel = nullptr);
int near_mma_prepare(pfft_plan *p, const std::vector<int64_t> &near_ptr, const std::vector<int32_t> &near_col,
                     cudaStream_t s);
int near_mma_launch(pfft_plan *p, int32_t R, cudaStream_t st);
// paired FP32 (y, z) plane convolution of ngrids x-transformed grids (static
// kernel); done = false when the plane size is not one it is built for
bool plane_conv_supported(const pfft_plan *p);
int plane_conv_f32(pfft_plan *p, float2 *spec, int32_t ngrids, cudaStream_t s, bool &done);
int check_device_errors(pfft_plan *p);
// Lossy kernel in pfft_matvec (sie_lossy.cu).  lossy_prepare: builds the per-frequency
// data missing for omega[R] (on stream st, synchronising it when something is built)
// and uploads the right-hand sides' slot tables; after it, lossy_sel / lossy_ltab
// describe this batch.  lossy_diag: the complex branch diagonal Lt_k[e][e] of each of
// the ns frequencies into out [ns][nb].
int lossy_prepare(pfft_plan *p, const double *omega, int32_t R, cudaStream_t st);
const SpecSel *lossy_sel(const pfft_plan *p, int prec);
const void *const *lossy_ltab(const pfft_plan *p, int prec);
const int32_t *lossy_rslot(const pfft_plan *p);
int lossy_diag(pfft_plan *p, const double *omega, int32_t ns, double2 *out, cudaStream_t st);
void plan_free_lossy(pfft_plan *p);
// Nested-dissection multifrontal LDL^T of the preconditioner's nodal Laplacian
// (sie_nd.cu): nd_build orders the nunk unknowns (adjacency uadj, positions
// xyz [nunk][3]) and builds the fronts, perm (new -> raw); nd_rows maps the
// Laplacian's row entries (new numbering) into their fronts; nd_factor
// factorises one frequency slot (admittances a [nb]) into L64 / L32 [sumL]
// through the workspace W [sumF]; nd_solve solves in place on u [R][nunk]
// with the factors L [nslots][sumL] of each right-hand side's slot and the
// update-vector workspace uv [R][sumU].
int nd_build(const std::vector<std::vector<int32_t>> &uadj, const std::vector<double> &xyz, std::vector<int32_t> &perm,
             NdState **out);
int nd_rows(NdState *s, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &row_oth);
int nd_factor(pfft_plan *p, NdState *s, const double2 *a, const int32_t *row_ptr, const int32_t *row_br, double2 *W,
              double2 *L64, float2 *L32, int *status, cudaStream_t st);
template <typename T>
int nd_solve(pfft_plan *p, const NdState *s, const C<T> *L, const int32_t *slot, const int32_t *grp, int32_t ngrp,
             C<T> *u, C<T> *uv, cudaStream_t st);
int nd_group_size();   // right-hand sides per solve group (grp rows)
int64_t nd_factor_size(const NdState *s);
int64_t nd_workspace_size(const NdState *s);
int64_t nd_update_size(const NdState *s);
void nd_info(const NdState *s, int32_t *fronts, int64_t *nnz, int32_t *max_front, int64_t *flops);
void nd_free(NdState *s);
// A port solve (Eq. LoopWithP) in steps (sie_solve.cu): gmres_create checks the
// arguments and sets up (workspace, right-hand sides, preconditioner factors,
// ||P^-1 b||) on stream st; gmres_top decides whether another cycle is needed;
// gmres_begin starts one; gmres_step enqueues one Arnoldi step (graph = true:
// every launch independent of the step index, for capture); after the stream
// has synchronised gmres_stepped tells whether the cycle is over; gmres_end
// closes the cycle (cont = false: the solve is over); gmres_finish extracts Z
// and the statistics and frees the run (gmres_free frees it otherwise).
struct GmresRun;
int gmres_create(pfft_plan *p, const double *freqs, int32_t nf, const int32_t *ports, int32_t np,
                 const sie_solve_opts *opts, cudaStream_t st, GmresRun **out);
int gmres_top(GmresRun *g, bool &need);
int gmres_begin(GmresRun *g);
int gmres_step(GmresRun *g, bool graph);
bool gmres_stepped(GmresRun *g);
int gmres_end(GmresRun *g, bool &cont);
int gmres_finish(GmresRun *g, sie_c64 *Z_out, sie_solve_stats *st_out);
void gmres_free(GmresRun *g);
cudaStream_t gmres_stream(const GmresRun *g);
int64_t gmres_plan_launches(const GmresRun *g);
// Complex padded table of exp(-jkR)/R (1/delta given) into Hc [Mx][My][Mz]; its folded
// spectrum scaled by 1/(Mx My Mz) into H64 / H32 (Hc may be overwritten).
int lossy_fill_table(pfft_plan *p, double inv_delta, double2 *Hc, cudaStream_t s);
int lossy_table_spectrum(pfft_plan *p, double2 *Hc, double2 *H64, float2 *H32, cudaStream_t s);
// End of a synchronous call on stream st: the error flags come back with the
// stream's one synchronisation (pinned copy) instead of a second round trip.
int finish_call(pfft_plan *p, cudaStream_t st);
}  // namespace sie
