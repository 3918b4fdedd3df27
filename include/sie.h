/*
 * sie.h - C ABI of the GB300 pFFT / loop-basis GMRES library (libsie).
 *
 * The library computes the port impedance of conductors described by a
 * triangle surface mesh with the magneto-quasi-static surface integral
 * equation of arXiv 2210.04891:
 *   Eq. (MPIE3)/(Zb): Z_b = Z_s G + (j w mu0 / 4 pi) Lt, branch = shared edge,
 *   Eq. (FinalME):    A Z_b A^T I_l = V_l in fundamental-loop space,
 *   Eq. (LoopWithP):  left-preconditioned GMRES with P = A diag(Z_b) A^T,
 *   Eq. (Lb):         Lt applied by the pre-corrected FFT, Lt ~ L_d + I H B.
 *
 * Conventions shared by every call
 *   - Units: metres, siemens per metre, hertz, radians per second, ohms.
 *   - Complex numbers are interleaved (re, im) pairs, FP64 unless stated.
 *   - Return value: SIE_OK (0) or a negative SIE_ERR_* code; nothing aborts
 *     or exits.  sie_last_error() gives a message for the calling thread.
 *   - Host input arrays are copied; the caller keeps ownership.  Handles are
 *     owned by the library and released by the matching *_destroy call
 *     (destroying NULL is a no-op).
 *   - Device pointers are CUDA device addresses on the device current when the
 *     plan was created.  `cuda_stream` is a cudaStream_t (NULL = legacy default
 *     stream); work is enqueued on it and the call returns when the results are
 *     ready unless stated otherwise.
 *   - A plan may be used by one thread at a time; separate plans are
 *     independent.
 */
#ifndef SIE_H
#define SIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SIE_OK = 0,
    SIE_ERR_ARG = -1,           /* invalid argument or size                      */
    SIE_ERR_NONMANIFOLD = -2,   /* an edge shared by more than two triangles     */
    SIE_ERR_BAD_PORT = -3,      /* empty contact, source == sink, or the two on
                                   separate conductors                           */
    SIE_ERR_OOM = -4,           /* host or device allocation failed              */
    SIE_ERR_CUDA = -5,          /* a CUDA call failed (message has the detail)   */
    SIE_ERR_NOT_CONVERGED = -6, /* GMRES hit its iteration cap                   */
    SIE_ERR_BREAKDOWN = -7,     /* zero pivot in the preconditioner or a
                                   non-finite value in the Krylov recurrence     */
    SIE_ERR_TIMEOUT = -8        /* a bounded device wait ran out                 */
};

enum { SIE_SPACE_LOOP = 0, SIE_SPACE_BRANCH = 1 };
enum { SIE_PREC_FP64 = 0, SIE_PREC_MIXED = 1, SIE_PREC_DF = 2 };
enum { SIE_KERNEL_STATIC = 0, SIE_KERNEL_LOSSY = 1 };

typedef struct sie_mesh sie_mesh;
typedef struct sie_loops sie_loops;
typedef struct pfft_plan pfft_plan;
typedef struct { double re, im; } sie_c64;

/* A port (Sec. III-C): a unit voltage source between two contact faces.
 * Each face is a set of triangle indices contracted into one circuit node. */
typedef struct {
    const int32_t *src;
    int32_t n_src;
    const int32_t *sink;
    int32_t n_sink;
} sie_port;

typedef struct {
    int64_t n_nodes;     /* circuit nodes after contact contraction            */
    int64_t n_branches;  /* b: edges shared by two triangles (port links not
                            counted)                                           */
    int64_t n_comp;      /* s: separate conductors                              */
    int64_t n_loops;     /* l = b - n + s + p (Sec. III-A, III-C)               */
    int64_t n_ports;     /* p                                                  */
    int64_t tree_depth;  /* depth of the breadth-first spanning forest         */
    int64_t nnz_A;       /* nonzeros of the loop matrix A (sum of loop lengths)*/
} sie_loop_stats;

/* pFFT parameters (Sec. IV-B leaves them open; these are the readings used). */
typedef struct {
    int32_t grid[3];       /* N_x, N_y, N_z grid nodes spanning the mesh box   */
    int32_t order;         /* stencil order O_s per axis, 2..4                 */
    double near_factor;    /* near radius = max(near_factor * max h,           */
    double near_min_diam;  /*                   near_min_diam * max diameter)  */
    int32_t n_touch;       /* outer Gauss order for pairs sharing a vertex     */
    int32_t kernel;        /* SIE_KERNEL_STATIC: 1/(4 pi R) (Eq. StaticGF);
                              SIE_KERNEL_LOSSY: exp(-j k R)/(4 pi R) of the
                              conductors' own conductivity (see pfft_matvec)  */
    double h0;             /* kernel value at zero grid offset (result does not
                              depend on it; kept for the independence check)   */
} pfft_params;

typedef struct {
    double tol;            /* preconditioned relative residual, e.g. 1e-6      */
    int32_t restart;       /* GMRES(m) restart length                          */
    int32_t max_iter;      /* iteration cap per right-hand side               */
    int32_t precond;       /* 0: none, 1: P = A diag(Z_b) A^T (Eq. Precond)    */
    int32_t prec;          /* SIE_PREC_FP64 or SIE_PREC_MIXED                  */
    int32_t refine;        /* with SIE_PREC_MIXED: 1 = iterative refinement:
                              every restart residual P^-1 (b - Z x) (and the
                              convergence test) in FP64, the Arnoldi cycles in
                              the mixed form; 2 = the same with the residual
                              products b - Z x in double-float (SIE_PREC_DF;
                              the norms stay FP64) and, where the
                              preconditioner takes the narrow band route, its
                              sweeps (inside the cycles and in the tests'
                              P^-1) in double-float; 0 = all in the mixed form */
} sie_solve_opts;

typedef struct {
    int32_t iterations_max;   /* largest iteration count over right-hand sides */
    int32_t iterations_sum;
    int32_t n_not_converged;
    double residual_max;      /* final preconditioned relative residual        */
    double seconds;           /* wall time of the solve phase                  */
    int64_t matvecs;          /* right-hand-side matvecs applied               */
} sie_solve_stats;

/* Mesh (Sec. II-B): nv vertices xyz[nv][3]; nt triangles tri[nt][3] whose
 * right-hand normal points out of the conductor; cond_id[nt] in [0, ncond);
 * sigma[ncond] > 0.  Errors: SIE_ERR_ARG for out-of-range indices, degenerate
 * triangles or non-positive conductivity. */
int sie_mesh_load(const double *xyz, int64_t nv, const int32_t *tri, int64_t nt,
                  const int32_t *cond_id, const double *sigma, int32_t ncond, sie_mesh **out);
/* The same mesh from a text file of this library's own format, version 1:
 *   sie_mesh 1
 *   <nv> <nt> <ncond>
 *   <sigma_0> ... <sigma_{ncond-1}>          (S/m)
 *   <x> <y> <z>                     nv lines (m)
 *   <v0> <v1> <v2> <cond_id>        nt lines (0-based vertex ids)
 * Tokens are separated by any whitespace; '#' starts a comment that runs to
 * the end of the line.  Numbers are read independently of the C locale; write
 * coordinates with 17 significant digits for an exact round trip.  Errors:
 * SIE_ERR_ARG (unreadable file, bad header, missing or malformed number,
 * trailing data, and every check of sie_mesh_load). */
int sie_mesh_load_file(const char *path, sie_mesh **out);
void sie_mesh_destroy(sie_mesh *m);

/* Circuit graph and fundamental loops (Sec. II-D, III): nodes = triangles
 * (contacts contracted), branches = shared edges oriented from the lower to the
 * higher triangle index, breadth-first spanning forest rooted at each part's
 * lowest node id, one loop per link, port links last.  `st` may be NULL.
 * Errors: SIE_ERR_NONMANIFOLD, SIE_ERR_BAD_PORT, SIE_ERR_ARG. */
int loop_basis_build(const sie_mesh *m, const sie_port *ports, int32_t np, sie_loops **out,
                     sie_loop_stats *st);
void sie_loops_destroy(sie_loops *l);

/* Export the loop matrix A (Eq. VolT) as CSR over loops: row_ptr[n_loops + 1],
 * col[nnz_A] (branch id; port p is column n_branches + p), val[nnz_A] (+1/-1),
 * columns of a row in the order the loop is walked.  Arrays are caller-owned
 * host memory of the sizes in sie_loop_stats; any pointer may be NULL to skip.
 * Also exports each branch's (T+, T-) pair when br_tri[2 * n_branches] != NULL. */
int sie_loops_export(const sie_loops *l, int64_t *row_ptr, int32_t *col, int8_t *val,
                     int32_t *br_tri);

/* Build the pFFT operator on the current device (Sec. IV-B): grid, stencils,
 * kernel spectrum, near list, closed-form near-field integrals minus the grid's
 * own near contribution (L_d = L_direct - (I H B)_near), Gram blocks and the
 * preconditioner's diagonal.  Allocates device memory for the plan's lifetime.
 * Errors: SIE_ERR_ARG (grid < 2 * order in an axis, order outside 2..4),
 * SIE_ERR_OOM, SIE_ERR_CUDA. */
int pfft_plan_create(const sie_mesh *m, const sie_loops *l, const pfft_params *p, void *cuda_stream,
                     pfft_plan **out);
void pfft_plan_destroy(pfft_plan *p);

/* Surface model of each conductor.  The paper's surface impedance (Eq.
 * ImpedanceOp) Z_s = (1 + j) / (sigma delta) assumes delta well below the
 * conductor's thickness; Sec. II-A names a thickness-aware model as the remedy
 * at low frequency.  With t_eff[c] > 0 conductor c uses the impedance of one
 * face of a slab of thickness t_eff[c]:
 *   Z_s = (gamma / sigma) coth(gamma t / 2),  gamma = (1 + j) / delta,
 * which equals the classic value to within 2 exp(-t / delta) when delta << t
 * and tends to the DC sheet value 2 / (sigma t) as omega -> 0.  For a bar of
 * cross-section w x t, t_eff = 2 w t / (2 (w + t)) (twice the area over the
 * perimeter) makes a uniform perimeter current carry the volume DC resistance
 * rho L / (w t); omega = 0 then has a solution (the classic model's loop system
 * is singular there).  t_eff = NULL or t_eff[c] = 0 selects the classic form.
 * Applies to every later pfft_matvec, pfft_precond_apply and sie_solve call of
 * the plan (cached preconditioner factors are rebuilt).  ncond must equal the
 * mesh's conductor count; thicknesses must be finite and >= 0 (SIE_ERR_ARG). */
int pfft_plan_set_surface_model(pfft_plan *p, const double *t_eff, int32_t ncond);

/* The product of Eq. (FinalME) for nrhs right-hand sides at once (Sec. IV-A/B):
 *   space = SIE_SPACE_LOOP:   y = A [Z_s G + c_L (L_d + I H B)] A^T x,
 *                              x, y device complex128 [nrhs][n_loops];
 *   space = SIE_SPACE_BRANCH: y = [Z_s G + c_L (L_d + I H B)] x,
 *                              x, y device complex128 [nrhs][n_branches];
 * with c_L = j w mu0 / (4 pi) and Z_s = (1 + j) sqrt(w mu0 / (2 sigma)) of each
 * conductor, w = omega[r] (host array, one angular frequency per right-hand
 * side).  prec = SIE_PREC_FP64 computes every step in FP64; SIE_PREC_MIXED runs
 * projection, FFT convolution, interpolation and the near field in FP32 (the
 * near field on the tensor cores for an even nrhs of at least 96, else on the
 * CUDA cores) and the loop/branch maps (prefix sums, branch differences, the
 * Z_s/c_L combination)
 * in double-float (FP32 pairs, about 48 significant bits); y is complex128 in
 * both.  SIE_PREC_DF computes every step in double-float on the FP32 pipes
 * (block records, twiddles and the kernel spectrum rounded once from FP64 to
 * double-float pairs, sums and products by the error-free two-sum and FMA
 * two-product): an FP64-class product (agreeing with SIE_PREC_FP64 to about
 * 1e-12 relative) at a fraction of its cost on a GPU whose FP64 rate is a small
 * share of its FP32 rate; static kernel only (SIE_ERR_ARG for a lossy plan);
 * the first call builds the double-float tables (about the size of the FP64
 * block records) on the plan's stream.  x and y must not overlap.  Scratch is
 * plan-owned and grown on demand (SIE_ERR_OOM if that fails).
 *
 * Plans created with pfft_params.kernel = SIE_KERNEL_LOSSY use the
 * lossy-conductor kernel exp(-j k R)/(4 pi R) in place of 1/(4 pi R) in the
 * inductive term and in all four pFFT steps, k = (1 - j)/delta with
 * delta = sqrt(2 / (w mu0 sigma)) the skin depth at each right-hand side's
 * w = omega[r] (> 0) and the conductors' conductivity (one value shared by
 * every conductor, else pfft_plan_create fails with SIE_ERR_ARG); the paper
 * states only the static kernel (Eq. StaticGF), this is the interior kernel of
 * the same MQS equations.  The direct near blocks are the static closed-form
 * blocks plus int int f.f' (exp(-jkR) - 1)/R by the product of the 7-point
 * Radon rule on both triangles (accurate while |k| times the panel diameter is
 * at most about one; beyond, the panels do not resolve the kernel).  Per
 * distinct w the plan builds and caches (up to 64 frequencies, least recently
 * used replaced) the complex kernel spectrum and the complex pre-corrected near
 * blocks, n_near x 9 x 24 bytes plus (N_x+1)(N_y+1)(N_z+1) x 24 bytes: the first
 * call with a new w synchronises cuda_stream and allocates.  The near field runs
 * on the CUDA cores in both precisions. */
int pfft_matvec(pfft_plan *p, const void *x, void *y, int32_t nrhs, const double *omega,
                int32_t space, int32_t prec, void *cuda_stream);

/* Apply the preconditioner of Eq. (Precond), z = P^-1 y with
 * P = A diag(Z_b) A^T (port links carry no impedance), for nrhs loop-space
 * vectors y, z (device complex128 [nrhs][n_loops]) at omega[r].  P is applied
 * through the nodal Laplacian of the same circuit, factorised (FP64) per
 * conductor on first use of each distinct omega set.  prec = SIE_PREC_FP64
 * runs every step in FP64; SIE_PREC_MIXED runs the drive, the triangular sweeps
 * on the rounded factor and the branch currents in FP32 (band width below 1024,
 * see pfft_precond_info; wider bands fall back to FP64); SIE_PREC_DF runs them
 * in double-float (factor rounded to FP32 pairs) where the band width is at most
 * 31 and in FP64 otherwise (an FP32 LDL^T solve of the nodal Laplacian, whose
 * condition grows with the mesh, keeps few correct digits).  The factor buffers and
 * the sweeps' scratch are stream-ordered allocations on cuda_stream from a
 * plan-owned memory pool.  omega[r] > 0, or 0 when every conductor has
 * a slab surface model (SIE_ERR_ARG otherwise).  Errors: SIE_ERR_BREAKDOWN for
 * a zero pivot. */
int pfft_precond_apply(pfft_plan *p, const void *y, void *z, int32_t nrhs, const double *omega,
                       int32_t prec, void *cuda_stream);

/* Structure of the preconditioner (built on first use, or by this call): band
 * width W of its banded LDL^T after the reverse Cuthill-McKee ordering (max
 * over blocks), unknowns, and blocks (one per connected group of unknowns).
 * The sweeps take warp-register tiles for W <= 31, one CTA per (right-hand
 * side, block) for 31 < W < 1024 (FP32 in the mixed form), and a one-warp FP64
 * sweep beyond.  Any pointer may be NULL. */
int pfft_precond_info(pfft_plan *p, int32_t *band_width, int64_t *unknowns, int64_t *blocks);

/* Factorisation route of the preconditioner (Eq. Precond asks for a direct
 * factorisation of P; it is applied through the nodal Laplacian of the same
 * circuit, see pfft_precond_apply):
 *   SIE_PC_AUTO  the band LDL^T after reverse Cuthill-McKee ordering when its
 *                band is below 1024, else nested dissection (the default);
 *   SIE_PC_BAND  always the band LDL^T;
 *   SIE_PC_ND    always nested dissection: the unknowns are bisected at the
 *                median of their positions along the longest axis, recursively
 *                (separators from the smaller side of each cut, leaves of at
 *                most 128 unknowns), and the Laplacian is factorised as a
 *                multifrontal LDL^T on the device (FP64; its FP32 rounding serves
 *                the mixed form's solves), fronts of one tree level at a time.
 * Setting a method drops the plan's preconditioner state (rebuilt on next use).
 * Errors: SIE_ERR_ARG for an unknown method. */
enum { SIE_PC_AUTO = 0, SIE_PC_BAND = 1, SIE_PC_ND = 2 };
int pfft_precond_set_method(pfft_plan *p, int32_t method);
/* Structure of a nested-dissection factorisation (built on first use, or by this
 * call): method_used (SIE_PC_BAND or SIE_PC_ND), fronts, nnz of the factor
 * (complex entries per frequency), largest front and complex multiply-adds of
 * one factorisation (all 0 for the band route).  Any pointer may be NULL. */
int pfft_precond_nd_info(pfft_plan *p, int32_t *method_used, int32_t *fronts, int64_t *nnz_factor,
                         int32_t *max_front, int64_t *flops);

/* Port impedance extraction (Sec. III-C, V): for every frequency f and every
 * port q a unit source in port q's loop, GMRES on Eq. (LoopWithP), then
 * Y[f][p][q] = loop current of port p, Z(f) = Y(f)^-1.  ports[np] selects the
 * plan's ports (indices into the ports given to loop_basis_build).
 * Z_out: caller-owned host [nf][np][np].  On SIE_ERR_NOT_CONVERGED Z_out and
 * st are still filled.  `st` may be NULL.  freqs[f] > 0, or f = 0 (DC: Z real)
 * when every conductor has a slab surface model (pfft_plan_set_surface_model);
 * SIE_ERR_ARG otherwise. */
int sie_solve(pfft_plan *p, const double *freqs, int32_t nf, const int32_t *ports, int32_t np,
              const sie_solve_opts *opts, sie_c64 *Z_out, sie_solve_stats *st);

/* Post-processing of loop currents x (device complex128 [nrhs][n_loops], e.g. a
 * solution of Eq. (LoopWithP)) into the quantities the paper plots (Sec. V):
 *   i_branch = A^T x                 branch currents (Eq. CurT), [nrhs][n_branches];
 *   v_branch = Z_b i_branch          voltage drops tail -> head (Eq. VolT, the
 *                                    SIE_SPACE_BRANCH product at omega[r]),
 *                                    [nrhs][n_branches];
 *   phi      = node potential of each panel, [nrhs][n_tri]: the sum of the
 *              tree-branch drops from the panel's node to its conductor's
 *              reference node (0 V), so v_branch = phi(tail) - phi(head) on
 *              every tree branch.  The reference node of a conductor is the
 *              sink contact of the first port on it, else its tree root;
 *              contact panels share their contact's potential.
 * All three outputs are caller-owned device complex128 buffers; any may be NULL
 * (not computed; temporaries are used where a later output needs it).  omega
 * (host, [nrhs]) is needed for v_branch or phi, may be NULL otherwise.  The
 * currents are exact FP64 sums; prec selects the product's arithmetic
 * (as in pfft_matvec); the potential sums are FP64.  Synchronises cuda_stream
 * before returning.  Errors: SIE_ERR_ARG (NULL x, nrhs < 1 or > 65535, bad
 * prec or omega), SIE_ERR_OOM, SIE_ERR_CUDA. */
int sie_postprocess(pfft_plan *p, const void *x, int32_t nrhs, const double *omega, int32_t prec,
                    void *i_branch, void *v_branch, void *phi, void *cuda_stream);

/* Batches of plans (uneven geometries solved together).  A batch borrows n
 * distinct plans on one device (each plan once) and owns a stream per plan;
 * while a batch call runs, the caller must not use its plans elsewhere.
 * Errors: SIE_ERR_ARG (NULL or repeated plan, plans on different devices),
 * SIE_ERR_CUDA, SIE_ERR_OOM. */
typedef struct sie_batch sie_batch;
int sie_batch_create(pfft_plan *const *plans, int32_t n, sie_batch **out);
void sie_batch_destroy(sie_batch *b);

/* The product of pfft_matvec for every plan i of the batch at once:
 * y[i] = (A) Z_b(omega[i][r]) (A^T) x[i], x[i], y[i] device complex128
 * [nrhs[i]][n_loops_i or n_branches_i]; omega[i] host [nrhs[i]]; space and prec
 * as in pfft_matvec, shared by all plans.  Each plan's kernels run on its own
 * stream, forked from cuda_stream and joined back (the call returns when every
 * result is ready).  use_graph = 1: the whole step, the per-plan coefficient
 * uploads (from pinned staging the batch owns) and every kernel, is captured
 * into one CUDA graph on the first call and replayed by later calls with the
 * same x, y, nrhs, space and prec (omega may change between replays); it is
 * captured again when any of these changes or a plan's scratch has been
 * reallocated.  Results equal pfft_matvec's bit for bit. */
int sie_batch_matvec(sie_batch *b, void *const *x, void *const *y, const int32_t *nrhs,
                     const double *const *omega, int32_t space, int32_t prec, int32_t use_graph,
                     void *cuda_stream);
/* Graph captures and replays so far (either pointer may be NULL). */
int sie_batch_stats(const sie_batch *b, int64_t *captures, int64_t *replays);

/* sie_solve for every plan i at once (one host thread per plan, each plan's
 * work on its batch stream): freqs[i][nf[i]], ports[i][np[i]], Z_out[i] host
 * [nf[i]][np[i]][np[i]], st_out[n] (may be NULL).  Returns the first plan's
 * error (message names the plan); every plan's Z and stats are still filled as
 * sie_solve fills them. */
int sie_batch_solve(sie_batch *b, const double *const *freqs, const int32_t *nf, const int32_t *const *ports,
                    const int32_t *np, const sie_solve_opts *opts, sie_c64 *const *Z_out,
                    sie_solve_stats *st_out);

/* sie_batch_solve with every plan's GMRES (Eq. LoopWithP) stepped in lockstep
 * under CUDA graph replay: the plans' set-ups (workspace, preconditioner
 * factors) and the ends of their restart cycles run concurrently on host
 * threads; within a cycle one Arnoldi step of every plan whose cycle is still
 * running (its product and preconditioner, classical Gram-Schmidt applied
 * twice, the Givens rotations and the convergence masks, all on the device,
 * the step index read on the device) is captured once into a graph on the
 * plans' streams and replayed with one launch per step; the graph is captured
 * again when a plan's cycle ends.  Per plan the arithmetic is that of sie_solve
 * (same kernels, same order), so Z and the statistics equal sie_solve's.
 * Arguments and errors as sie_batch_solve. */
int sie_batch_solve_graph(sie_batch *b, const double *const *freqs, const int32_t *nf, const int32_t *const *ports,
                          const int32_t *np, const sie_solve_opts *opts, sie_c64 *const *Z_out,
                          sie_solve_stats *st_out);

/* Grid autotuning.  Candidates: the base grid, half and double it on every
 * axis, and the base with one axis doubled (axes kept within the plan's size
 * rules, at most SIE_TUNE_MAX).  Each is built, its FP64 loop-space product of
 * nrhs fixed pseudo-random vectors at omega compared with that of the finest
 * candidate built with 1.5 x base->near_factor (the reference; relative 2-norm,
 * max over right-hand sides), and its mixed matvec timed with CUDA events on
 * cuda_stream (5 after 2 warm-ups).  best = the fastest candidate within tol
 * of the reference (else the reference's grid and radius); `rep` (may be NULL)
 * gets every candidate's grid, time and error.  Builds and frees one plan at a
 * time.  Errors: SIE_ERR_ARG, and those of pfft_plan_create / pfft_matvec. */
#define SIE_TUNE_MAX 8
typedef struct {
    int32_t n_tried;
    int32_t best;                   /* index of the chosen candidate, -1 if none was within tol */
    int32_t grid[SIE_TUNE_MAX][3];
    double ms[SIE_TUNE_MAX];        /* mixed matvec time, milliseconds */
    double err[SIE_TUNE_MAX];       /* relative difference to the reference */
} sie_tune_report;
int pfft_autotune(const sie_mesh *m, const sie_loops *l, const pfft_params *base, int32_t nrhs, double omega,
                  double tol, void *cuda_stream, pfft_params *best, sie_tune_report *rep);

/* Kernel launch shapes of a plan's product (none changes the result beyond the
 * rounding of the near-field path in the mixed form):
 *   near      0: automatic (mixed form: tensor cores for an even right-hand-side
 *                count of at least 96, else the CUDA-core gather);
 *             1: tensor cores for any even count (mixed form);
 *             2: the CUDA-core gather;
 *   far_slab  right-hand sides per warp in the mixed far-field gather, 64 or 128
 *             (0: 64);
 *   proj_slab the projection: 32 = node chunks with their triangles' currents
 *             staged in shared memory, 32 right-hand sides per slab (mixed
 *             form); 64 or 128 = right-hand sides per warp of the direct
 *             gather (0: 128);
 *   plane_gpc grids per CTA in the (y, z) plane kernel, 1..8 (0: up to 8, as
 *             many as keep about four waves).
 * Errors: SIE_ERR_ARG for a value outside these. */
typedef struct {
    int32_t near;
    int32_t far_slab;
    int32_t proj_slab;
    int32_t plane_gpc;
} sie_kernel_tuning;
int pfft_plan_set_kernel_tuning(pfft_plan *p, const sie_kernel_tuning *t);   /* NULL: all automatic */
int pfft_plan_get_kernel_tuning(const pfft_plan *p, sie_kernel_tuning *t);

/* Kernel autotuning of a plan: its mixed loop-space product at nrhs right-hand
 * sides and omega timed with CUDA events on cuda_stream (5 products after 2
 * warm-ups) for every combination of near path (automatic and the other
 * applicable one), far-field slab (64, 128), projection (32, 64, 128) and
 * plane grids per CTA (automatic, 4); the fastest is set on the plan and
 * returned in best; rep (may be NULL) gets every candidate and its time.
 * Errors: those of pfft_matvec. */
#define SIE_KTUNE_MAX 32
typedef struct {
    int32_t n_tried;
    int32_t best;
    sie_kernel_tuning cand[SIE_KTUNE_MAX];
    double ms[SIE_KTUNE_MAX];
} sie_kernel_tune_report;
int pfft_autotune_kernels(pfft_plan *p, int32_t nrhs, double omega, void *cuda_stream, sie_kernel_tuning *best,
                          sie_kernel_tune_report *rep);

/* Learned correction of the preconditioner (Eq. Precond): D'_e = D_e (1 + g(f_e))
 * for the diagonal D_e of Z_b on each branch, g a network of six per-branch
 * features at the frequency (quarter decades of |Z_s| G_ee, c_L Lt_ee, their
 * ratio, G_ee, Lt_ee and omega), f [6] -> tanh [H] -> tanh [H] ->
 * g = 0.5 tanh(.), H = 16 or 32 (FP32 parameters) or 128 (the network computes
 * with FP16 roundings of FP32 master parameters, FP32 accumulation; Adam
 * updates the masters), parameters on the device, flat
 * [W1 H x 6][b1 H][W2 H x H][b2 H][w3 H][b3].  A new network has a zero output
 * layer: g = 0, the plain preconditioner.  Training is full-batch mean squared
 * error against per-branch targets with Adam (device kernels); the plain
 * preconditioner stays the fallback (pfft_plan_set_learned(p, NULL)).
 * Errors: SIE_ERR_ARG, SIE_ERR_OOM, SIE_ERR_CUDA. */
typedef struct sie_mlp sie_mlp;
int sie_mlp_create(int32_t hidden, uint64_t seed, sie_mlp **out);
void sie_mlp_destroy(sie_mlp *m);
int64_t sie_mlp_param_count(const sie_mlp *m);
int sie_mlp_get_params(const sie_mlp *m, float *host, int64_t n);
int sie_mlp_set_params(sie_mlp *m, const float *host, int64_t n);   /* also resets Adam's moments */
/* g [n] (device float) of features [n][6] (device float); synchronises cuda_stream. */
int sie_mlp_forward(const sie_mlp *m, const float *feats, int64_t n, float *g, void *cuda_stream);
/* Gradient (host [param_count], may be NULL) and loss (host, may be NULL) of the
 * mean squared error (1/n) sum (g_e - t_e)^2, features and targets on the device. */
int sie_mlp_grad(sie_mlp *m, const float *feats, const float *target, int64_t n, float *grad_host,
                 float *loss_host, void *cuda_stream);
/* `steps` Adam steps (lr; moments persist across calls); loss before each step into
 * loss_host [steps] (may be NULL). */
int sie_mlp_train(sie_mlp *m, const float *feats, const float *target, int64_t n, int32_t steps, float lr,
                  float *loss_host, void *cuda_stream);
/* Features of every branch of the plan at omega: feats device float [n_branches][6]. */
int pfft_branch_features(pfft_plan *p, double omega, float *feats, void *cuda_stream);
/* Training target per branch: t_e = sum_k Re(conj(D_e a_ke) (Z_b a_k)_e) / sum_k |D_e a_ke|^2 - 1,
 * clipped to [-0.45, 0.45], for k probe branch currents alpha (device complex128
 * [k][n_branches]) at omega; Z_b a_k is the branch-space product (FP64).
 * target: device float [n_branches]. */
int pfft_branch_probe_target(pfft_plan *p, const void *alpha, int32_t k, double omega, float *target,
                             void *cuda_stream);
/* Use the network (borrowed: keep it alive while set) in the plan's preconditioner,
 * or NULL for the plain one; cached factors are rebuilt on next use. */
int pfft_plan_set_learned(pfft_plan *p, const sie_mlp *m);

/* Self-test of failure detection: a one-thread kernel waits, with the bounded
 * wait the tensor-core near field uses (mbarrier try_wait under a time limit),
 * on a barrier nothing completes; the wait runs out after limit_ms (<= 1000),
 * sets the plan's device error flag and returns, and the call reads the flag
 * back as the library's calls do.  Expected result: SIE_ERR_TIMEOUT, with the
 * flag cleared and the plan and its CUDA context usable; SIE_OK would mean the
 * wait never ran out.  No fault, trap or hang is involved. */
int sie_selftest_bounded_wait(pfft_plan *p, double limit_ms, void *cuda_stream);

/* Plan introspection for tests and benchmarks: sizes (any pointer may be NULL). */
int pfft_plan_info(const pfft_plan *p, int64_t *n_loops, int64_t *n_branches, int64_t *n_tri,
                   int64_t *n_near_pairs, double *grid_h /* [3] */, double *r_near,
                   int64_t *device_bytes);

/* Copy one of the plan's setup arrays to caller-owned host memory (for checks):
 *   SIE_EXPORT_NEAR_PTR  int64  [n_tri + 1]   near-list row offsets (rows = triangles)
 *   SIE_EXPORT_NEAR_COL  int32  [n_near]      near triangles of each row, ascending
 *   SIE_EXPORT_LD        double [n_near][3][3] pre-corrected blocks L_direct - (I H B)
 *   SIE_EXPORT_LDIRECT   double [n_near][3][3] direct blocks
 *   SIE_EXPORT_HHAT      double [N_y+1][N_z+1][N_x+1] kernel spectrum / (8 N_x N_y N_z),
 *                        index k folded to min(k, 2N - k) per axis
 *   SIE_EXPORT_START     int32  [n_tri][7][3] stencil start node of each sample point
 *   SIE_EXPORT_PROJ_PTR  int64  [n_tri + 1]   projection-block row offsets (rows = triangles);
 *                        the last entry is the number of (node, triangle) pairs n_pair
 *   SIE_EXPORT_PROJ_NODE int32  [n_pair]      grid node n of each block, ascending per row
 *   SIE_EXPORT_PROJ_W    double [n_pair][3][3] W(n, T)[d][k] = sum_q L_n(r_q) (w_q/2)(r_q - v_k)_d,
 *                        the projection of Sec. IV-B with the point currents folded in
 * capacity_bytes is the size of host_out; SIE_ERR_ARG if it is too small. */
enum { SIE_EXPORT_NEAR_PTR = 0, SIE_EXPORT_NEAR_COL = 1, SIE_EXPORT_LD = 2, SIE_EXPORT_LDIRECT = 3,
       SIE_EXPORT_HHAT = 4, SIE_EXPORT_START = 5, SIE_EXPORT_PROJ_PTR = 6, SIE_EXPORT_PROJ_NODE = 7,
       SIE_EXPORT_PROJ_W = 8 };
int pfft_plan_export(const pfft_plan *p, int32_t what, void *host_out, int64_t capacity_bytes);

/* Step 2 of Sec. IV-B alone: phi_g = H Q_g for nbatch grids, in place.
 * grid: device [nbatch][N_x][N_y][N_z] complex (complex128 for SIE_PREC_FP64,
 * complex64 for SIE_PREC_MIXED), node (i, j, k) at h-spaced offsets from the
 * mesh box's low corner.  Aperiodic convolution with H(d) = 1/|d o h| (h0 at
 * d = 0) via the zero-padded FFT. */
int pfft_convolve(pfft_plan *p, void *grid, int32_t nbatch, int32_t prec, void *cuda_stream);

/* Step 2 of Sec. IV-B with the lossy-conductor kernel instead of the static one:
 * phi_g = H_k Q_g with H_k(d) = exp(-j k R) / R, R = |d o h| (h0 at d = 0),
 * k = (1 - j) / delta and delta = sqrt(2 / (omega mu0 sigma)) the skin depth,
 * in the e^{j w t} convention of Z_s (Eq. ImpedanceOp), so |H_k| decays as
 * exp(-R / delta) and H_k -> 1/R as omega -> 0.  The paper states only the
 * static Green's function (Eq. StaticGF); this is the interior-region kernel of
 * the same MQS equations, for lossy-region variants of the method.  Grids,
 * layout and padding as pfft_convolve (nbatch grids, in place).  The complex
 * kernel spectrum is built (FP64) on first use of an (omega, sigma) pair and
 * kept until another pair is asked for.  Errors: SIE_ERR_ARG for omega or sigma
 * not finite and positive. */
int pfft_convolve_lossy(pfft_plan *p, void *grid, int32_t nbatch, double omega, double sigma, int32_t prec,
                        void *cuda_stream);

/* pfft_convolve without any device allocation (the paper has no counterpart;
 * this is an interface for callers that may not allocate device memory when
 * they convolve: fixed start-up memory budgets, real-time loops that cannot
 * take cudaMalloc's synchronisation and latency, frameworks that own the
 * allocator).  Same arguments and result as pfft_convolve.  Its scratch is one
 * file-scope device array of 4 MiB that every GPU loading the library holds
 * until exit.  One grid needs, in values of the precision (16 B FP64, 8 B
 * mixed): 2N_x * N_y * N_z (the copy zero-padded along x) when its padded
 * (y, z) plane fits one CTA, and 2N_x * (N_y + 2N_y) * N_z (that copy and its
 * y transform) when it does not (2N_y * 2N_z > 8192, N_y or N_z above 128,
 * or 3 N_y (2N_z + 1) FP64 complex values above 200 KiB); a grid needing more
 * than 4 MiB is rejected with SIE_ERR_ARG.
 * Larger batches are processed in pieces that fit.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, with that device
 * current) and keeps it with the id of the device's context; a later call in
 * a new context (after cudaDeviceReset) looks it up again.  Make the first
 * call on each device before any stream capture.  The call synchronises cuda_stream
 * before it returns.  All calls share the one array, so calls that overlap on
 * the GPU (other streams, other host threads) race and corrupt each other's
 * results; nothing in the array needs clearing between calls. */
int pfft_convolve_noalloc(pfft_plan *p, void *grid, int32_t nbatch, int32_t prec, void *cuda_stream);

/* Stage timing (tracing).  When enabled, every stage of pfft_matvec,
 * pfft_precond_apply and sie_solve is bracketed by CUDA events recorded on the
 * stream the stage runs on; pfft_profile_read waits for them and returns the
 * accumulated device time (ms) and launch count of each stage since the last
 * enable.  Disabled by default; enabling resets the counters.  In pfft_matvec:
 *   LOOP_TO_BRANCH  loop currents -> local edge currents c_T (A^T, Euler-tour scan)
 *   POINT_CURRENTS  not launched: the point currents are folded into the projection blocks
 *   PROJECT         grid currents Q_g = sum_T W(n, T) c_T (Sec. IV-B step 1)
 *   FFT_X_FWD       phi_g = H Q_g (step 2): x pencils forward (zero-padded along x)
 *   FFT_YZ          per x-frequency plane: zero-padded y/z transform, kernel product,
 *                   inverse y/z transform, crop
 *   FFT_X_INV       x pencils inverse, crop
 *   INTERP          grid potentials regrouped with the right-hand sides innermost
 *   NEAR            per triangle: pre-corrected near blocks (step 4) + interpolation
 *                   (step 3) + Z_s Gram term, one fused gather
 *   BRANCH_TO_LOOP  triangle outputs -> branch voltages -> loop voltages (A) */
enum { SIE_STAGE_LOOP_TO_BRANCH = 0, SIE_STAGE_POINT_CURRENTS = 1, SIE_STAGE_PROJECT = 2,
       SIE_STAGE_FFT_X_FWD = 3, SIE_STAGE_FFT_YZ = 4, SIE_STAGE_FFT_X_INV = 5,
       SIE_STAGE_INTERP = 6, SIE_STAGE_NEAR = 7, SIE_STAGE_BRANCH_TO_LOOP = 8,
       SIE_STAGE_PRECOND_APPLY = 9, SIE_STAGE_PRECOND_FACTOR = 10, SIE_STAGE_ARNOLDI = 11,
       SIE_NSTAGES = 12 };
int pfft_profile_enable(pfft_plan *p, int32_t on);
int pfft_profile_read(pfft_plan *p, double *ms /* [SIE_NSTAGES] */, int64_t *launches /* [SIE_NSTAGES] */);

/* Number of this library's kernel launches since the plan was created. */
int64_t pfft_plan_launches(const pfft_plan *p);

const char *sie_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SIE_H */
