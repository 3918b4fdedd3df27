// Batched uneven geometries: many plans (one per geometry, each with its own
// grid, near field and loop basis) driven together.
//
// sie_batch_matvec runs every plan's product (Sec. IV-B steps 1-4 and the loop
// maps) on a stream of its own, forked from the caller's stream and joined
// back, so that the small kernels of many small geometries overlap on the GPU.
// With graphs enabled, the whole multi-plan step (coefficient uploads from
// pinned staging plus every kernel of every plan) is captured once into a CUDA
// graph and then replayed with one launch per step; the graph is captured
// again when an input address, a right-hand-side count, the space or the
// precision changes, or when a plan's scratch has been reallocated.
// sie_batch_solve runs the plans' port solves (Sec. III-C, IV-A) concurrently,
// one host thread per plan on the plan's batch stream.
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "sie_plan.h"

using namespace sie;

struct sie_batch {
    std::vector<pfft_plan *> plans;
    std::vector<cudaStream_t> streams;   // one per plan, non-blocking
    std::vector<cudaEvent_t> done;       // join events, one per plan
    cudaStream_t origin = nullptr;       // capture origin
    cudaEvent_t fork = nullptr;
    int device = 0;
    // pinned coefficient staging per plan: [cap][2 ncond + 1] FP64, then the float2 copy
    std::vector<void *> h_coef;
    std::vector<int32_t> h_cap;
    // graph cache
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key_x;
    std::vector<void *> key_y;
    std::vector<int32_t> key_r;
    std::vector<uint64_t> key_gen;
    int32_t key_space = -1, key_prec = -1;
    std::vector<int64_t> graph_launches;   // kernels per plan in one replay
    int64_t captures = 0, replays = 0;
};

namespace {

int ensure_staging(sie_batch *b, size_t i, int32_t R) {
    if (b->h_cap[i] >= R) return SIE_OK;
    if (b->h_coef[i]) cudaFreeHost(b->h_coef[i]);
    b->h_coef[i] = nullptr;
    b->h_cap[i] = 0;
    const size_t n = size_t(R) * (2 * b->plans[i]->ncond + 1);
    if (cudaMallocHost(&b->h_coef[i], n * (sizeof(double) + sizeof(float2))) != cudaSuccess)
        return fail(SIE_ERR_OOM, "sie_batch: pinned host allocation failed");
    b->h_cap[i] = R;
    return SIE_OK;
}

void drop_graph(sie_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->key_x.clear();
}

bool key_matches(const sie_batch *b, void *const *x, void *const *y, const int32_t *nrhs, int32_t space,
                 int32_t prec) {
    if (!b->exec || b->key_space != space || b->key_prec != prec) return false;
    for (size_t i = 0; i < b->plans.size(); ++i)
        if (b->key_x[i] != x[i] || b->key_y[i] != y[i] || b->key_r[i] != nrhs[i] ||
            b->key_gen[i] != b->plans[i]->scr_gen)
            return false;
    return true;
}

// Coefficients of plan i into its pinned staging (host work, before a launch).
int stage_coef(sie_batch *b, size_t i, const double *omega, int32_t R) {
    pfft_plan *p = b->plans[i];
    const size_t n = size_t(R) * (2 * p->ncond + 1);
    double *cf = static_cast<double *>(b->h_coef[i]);
    float2 *cd = reinterpret_cast<float2 *>(cf + size_t(b->h_cap[i]) * (2 * p->ncond + 1));
    (void)n;
    return fill_coef(p, omega, R, cf, cd);
}

// Enqueue the whole multi-plan step on the origin stream (captured).
int enqueue_step(sie_batch *b, void *const *x, void *const *y, const int32_t *nrhs, int32_t space, int32_t prec) {
    SIE_CUDA(cudaEventRecord(b->fork, b->origin));
    for (size_t i = 0; i < b->plans.size(); ++i) {
        pfft_plan *p = b->plans[i];
        cudaStream_t st = b->streams[i];
        SIE_CUDA(cudaStreamWaitEvent(st, b->fork, 0));
        const size_t n = size_t(nrhs[i]) * (2 * p->ncond + 1);
        const double *cf = static_cast<const double *>(b->h_coef[i]);
        const float2 *cd = reinterpret_cast<const float2 *>(cf + size_t(b->h_cap[i]) * (2 * p->ncond + 1));
        SIE_CUDA(cudaMemcpyAsync(p->scr.coef, cf, n * sizeof(double), cudaMemcpyHostToDevice, st));
        SIE_CUDA(cudaMemcpyAsync(coef_dd(p), cd, n * sizeof(float2), cudaMemcpyHostToDevice, st));
        const int64_t before = p->launches;
        int rc = matvec_launch(p, x[i], y[i], nrhs[i], space, prec, st);
        if (rc) return rc;
        b->graph_launches[i] = p->launches - before;
        SIE_CUDA(cudaEventRecord(b->done[i], st));
        SIE_CUDA(cudaStreamWaitEvent(b->origin, b->done[i], 0));
    }
    return SIE_OK;
}

int capture(sie_batch *b, void *const *x, void *const *y, const int32_t *nrhs, int32_t space, int32_t prec) {
    drop_graph(b);
    // stage timers record events, which a graph cannot hand back: off while capturing
    std::vector<bool> prof(b->plans.size());
    for (size_t i = 0; i < b->plans.size(); ++i) {
        prof[i] = b->plans[i]->prof_on;
        b->plans[i]->prof_on = false;
    }
    auto restore = [&]() {
        for (size_t i = 0; i < b->plans.size(); ++i) b->plans[i]->prof_on = prof[i];
    };
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        restore();
        return fail(SIE_ERR_CUDA, std::string("sie_batch: cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    }
    const int rc = enqueue_step(b, x, y, nrhs, space, prec);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->origin, &graph);
    restore();
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        return rc ? rc : fail(SIE_ERR_CUDA, std::string("sie_batch: capture failed: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return fail(SIE_ERR_CUDA, std::string("sie_batch: cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    const size_t n = b->plans.size();
    b->key_x.assign(x, x + n);
    b->key_y.assign(y, y + n);
    b->key_r.assign(nrhs, nrhs + n);
    b->key_gen.resize(n);
    for (size_t i = 0; i < n; ++i) b->key_gen[i] = b->plans[i]->scr_gen;
    b->key_space = space;
    b->key_prec = prec;
    ++b->captures;
    return SIE_OK;
}

}  // namespace

extern "C" int sie_batch_create(pfft_plan *const *plans, int32_t n, sie_batch **out) {
    if (!out) return fail(SIE_ERR_ARG, "sie_batch_create: out is NULL");
    *out = nullptr;
    if (!plans || n < 1) return fail(SIE_ERR_ARG, "sie_batch_create: no plans");
    for (int32_t i = 0; i < n; ++i) {
        if (!plans[i]) return fail(SIE_ERR_ARG, "sie_batch_create: NULL plan");
        if (plans[i]->device != plans[0]->device) return fail(SIE_ERR_ARG, "sie_batch_create: plans on different devices");
        if (plans[i]->params.kernel != SIE_KERNEL_STATIC)
            return fail(SIE_ERR_ARG, "sie_batch_create: batches take plans of the static kernel");
        for (int32_t j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return fail(SIE_ERR_ARG, "sie_batch_create: a plan appears twice");
    }
    sie_batch *b = new (std::nothrow) sie_batch;
    if (!b) return fail(SIE_ERR_OOM, "sie_batch_create: out of host memory");
    b->plans.assign(plans, plans + n);
    b->device = plans[0]->device;
    b->h_coef.assign(n, nullptr);
    b->h_cap.assign(n, 0);
    b->graph_launches.assign(n, 0);
    auto bail = [&](const char *what, cudaError_t e) {
        sie_batch_destroy(b);
        return fail(SIE_ERR_CUDA, std::string("sie_batch_create: ") + what + ": " + cudaGetErrorString(e));
    };
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bail("cudaSetDevice", e);
    if ((e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream", e);
    if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) return bail("event", e);
    b->streams.assign(n, nullptr);
    b->done.assign(n, nullptr);
    for (int32_t i = 0; i < n; ++i) {
        if ((e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking)) != cudaSuccess) return bail("stream", e);
        if ((e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming)) != cudaSuccess) return bail("event", e);
    }
    *out = b;
    return SIE_OK;
}

extern "C" void sie_batch_destroy(sie_batch *b) {
    if (!b) return;
    drop_graph(b);
    for (auto s : b->streams) if (s) cudaStreamDestroy(s);
    for (auto e : b->done) if (e) cudaEventDestroy(e);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->fork) cudaEventDestroy(b->fork);
    for (void *h : b->h_coef) if (h) cudaFreeHost(h);
    delete b;
}

extern "C" int sie_batch_matvec(sie_batch *b, void *const *x, void *const *y, const int32_t *nrhs,
                                const double *const *omega, int32_t space, int32_t prec, int32_t use_graph,
                                void *cuda_stream) {
    if (!b || !x || !y || !nrhs || !omega) return fail(SIE_ERR_ARG, "sie_batch_matvec: NULL argument");
    if (space != SIE_SPACE_LOOP && space != SIE_SPACE_BRANCH) return fail(SIE_ERR_ARG, "sie_batch_matvec: bad space");
    if (prec != SIE_PREC_FP64 && prec != SIE_PREC_MIXED) return fail(SIE_ERR_ARG, "sie_batch_matvec: bad precision");
    const size_t n = b->plans.size();
    for (size_t i = 0; i < n; ++i) {
        if (!x[i] || !y[i] || !omega[i] || nrhs[i] < 1)
            return fail(SIE_ERR_ARG, "sie_batch_matvec: bad input for plan " + std::to_string(i));
        const int64_t len = space == SIE_SPACE_LOOP ? b->plans[i]->nl : b->plans[i]->nb;
        const size_t bytes = size_t(nrhs[i]) * len * sizeof(double2);
        const char *xb = static_cast<const char *>(x[i]), *yb = static_cast<const char *>(y[i]);
        if (xb < yb + bytes && yb < xb + bytes) return fail(SIE_ERR_ARG, "sie_batch_matvec: x and y overlap");
    }
    cudaStream_t caller = static_cast<cudaStream_t>(cuda_stream);
    (void)cudaGetLastError();
    SIE_CUDA(cudaSetDevice(b->device));
    int rc;
    for (size_t i = 0; i < n; ++i)
        if ((rc = scratch_reserve(b->plans[i], nrhs[i], prec))) return rc;
    if (!use_graph) {
        SIE_CUDA(cudaEventRecord(b->fork, caller));
        for (size_t i = 0; i < n; ++i) {
            SIE_CUDA(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
            if ((rc = matvec_async(b->plans[i], x[i], y[i], nrhs[i], omega[i], space, prec, b->streams[i]))) return rc;
            SIE_CUDA(cudaEventRecord(b->done[i], b->streams[i]));
            SIE_CUDA(cudaStreamWaitEvent(caller, b->done[i], 0));
        }
    } else {
        for (size_t i = 0; i < n; ++i) {
            if ((rc = ensure_staging(b, i, nrhs[i]))) return rc;
            if ((rc = stage_coef(b, i, omega[i], nrhs[i]))) return rc;
        }
        if (!key_matches(b, x, y, nrhs, space, prec)) {
            // kernels' shared-memory attributes are set by an eager pass before the capture
            SIE_CUDA(cudaEventRecord(b->fork, caller));
            SIE_CUDA(cudaStreamWaitEvent(b->origin, b->fork, 0));
            if ((rc = enqueue_step(b, x, y, nrhs, space, prec))) return rc;
            SIE_CUDA(cudaStreamSynchronize(b->origin));
            if ((rc = capture(b, x, y, nrhs, space, prec))) return rc;
        }
        SIE_CUDA(cudaGraphLaunch(b->exec, caller));
        for (size_t i = 0; i < n; ++i) b->plans[i]->launches += b->graph_launches[i];
        ++b->replays;
    }
    SIE_CUDA(cudaStreamSynchronize(caller));
    for (size_t i = 0; i < n; ++i)
        if ((rc = check_device_errors(b->plans[i]))) return rc;
    return SIE_OK;
}

extern "C" int sie_batch_stats(const sie_batch *b, int64_t *captures, int64_t *replays) {
    if (!b) return fail(SIE_ERR_ARG, "sie_batch_stats: NULL batch");
    if (captures) *captures = b->captures;
    if (replays) *replays = b->replays;
    return SIE_OK;
}

extern "C" int sie_batch_solve(sie_batch *b, const double *const *freqs, const int32_t *nf,
                               const int32_t *const *ports, const int32_t *np, const sie_solve_opts *opts,
                               sie_c64 *const *Z_out, sie_solve_stats *st_out) {
    if (!b || !freqs || !nf || !ports || !np || !opts || !Z_out) return fail(SIE_ERR_ARG, "sie_batch_solve: NULL argument");
    const size_t n = b->plans.size();
    std::vector<int> rcs(n, SIE_OK);
    std::vector<std::string> msgs(n);
    std::vector<std::thread> workers;
    workers.reserve(n);
    for (size_t i = 0; i < n; ++i) {
        workers.emplace_back([&, i]() {
            pfft_plan *p = b->plans[i];
            if (cudaSetDevice(b->device) != cudaSuccess) {
                rcs[i] = SIE_ERR_CUDA;
                msgs[i] = "cudaSetDevice failed";
                return;
            }
            cudaStream_t own = p->stream;
            p->stream = b->streams[i];   // the plan's solve on its batch stream
            rcs[i] = sie_solve(p, freqs[i], nf[i], ports[i], np[i], opts, Z_out[i], st_out ? &st_out[i] : nullptr);
            p->stream = own;
            if (rcs[i]) msgs[i] = sie_last_error();
        });
    }
    for (auto &t : workers) t.join();
    for (size_t i = 0; i < n; ++i)
        if (rcs[i]) return fail(rcs[i], "sie_batch_solve: plan " + std::to_string(i) + ": " + msgs[i]);
    return SIE_OK;
}

namespace {

// Runs fn(i) for i in [0, n) on one host thread each (the plans' set-ups and
// cycle ends synchronise their own streams; threads let them overlap).
template <typename F>
void each_plan(sie_batch *b, const std::vector<size_t> &which, F fn) {
    std::vector<std::thread> th;
    th.reserve(which.size());
    for (size_t i : which)
        th.emplace_back([&, i]() {
            cudaSetDevice(b->device);
            fn(i);
        });
    for (auto &t : th) t.join();
}

// One Arnoldi step of every run in `set`, each on its plan's batch stream,
// forked from and joined back into the origin stream.
int enqueue_gmres_step(sie_batch *b, const std::vector<GmresRun *> &runs, const std::vector<size_t> &set,
                       std::vector<int64_t> &launches) {
    SIE_CUDA(cudaEventRecord(b->fork, b->origin));
    for (size_t i : set) {
        SIE_CUDA(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
        const int64_t before = gmres_plan_launches(runs[i]);
        int rc = gmres_step(runs[i], true);
        if (rc) return rc;
        launches[i] = gmres_plan_launches(runs[i]) - before;
        SIE_CUDA(cudaEventRecord(b->done[i], b->streams[i]));
        SIE_CUDA(cudaStreamWaitEvent(b->origin, b->done[i], 0));
    }
    return SIE_OK;
}

int capture_gmres_step(sie_batch *b, const std::vector<GmresRun *> &runs, const std::vector<size_t> &set,
                       std::vector<int64_t> &launches, cudaGraphExec_t *exec) {
    *exec = nullptr;
    std::vector<bool> prof(b->plans.size());
    for (size_t i = 0; i < b->plans.size(); ++i) {
        prof[i] = b->plans[i]->prof_on;
        b->plans[i]->prof_on = false;
    }
    auto restore = [&]() {
        for (size_t i = 0; i < b->plans.size(); ++i) b->plans[i]->prof_on = prof[i];
    };
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        restore();
        return fail(SIE_ERR_CUDA, std::string("sie_batch_solve_graph: cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    }
    const int rc = enqueue_gmres_step(b, runs, set, launches);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->origin, &graph);
    restore();
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        return rc ? rc : fail(SIE_ERR_CUDA, std::string("sie_batch_solve_graph: capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *exec = nullptr;
        return fail(SIE_ERR_CUDA, std::string("sie_batch_solve_graph: cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    ++b->captures;
    return SIE_OK;
}

}  // namespace

extern "C" int sie_batch_solve_graph(sie_batch *b, const double *const *freqs, const int32_t *nf,
                                     const int32_t *const *ports, const int32_t *np, const sie_solve_opts *opts,
                                     sie_c64 *const *Z_out, sie_solve_stats *st_out) {
    if (!b || !freqs || !nf || !ports || !np || !opts || !Z_out)
        return fail(SIE_ERR_ARG, "sie_batch_solve_graph: NULL argument");
    const size_t n = b->plans.size();
    SIE_CUDA(cudaSetDevice(b->device));
    (void)cudaGetLastError();
    std::vector<GmresRun *> runs(n, nullptr);
    std::vector<int> rcs(n, SIE_OK);
    std::vector<std::string> msgs(n);
    std::vector<size_t> all(n);
    for (size_t i = 0; i < n; ++i) all[i] = i;
    auto first_error = [&](const char *what) -> int {
        for (size_t i = 0; i < n; ++i)
            if (rcs[i]) return fail(rcs[i], std::string("sie_batch_solve_graph: ") + what + " of plan " +
                                                std::to_string(i) + ": " + msgs[i]);
        return SIE_OK;
    };
    auto cleanup = [&]() {
        for (GmresRun *g : runs)
            if (g) gmres_free(g);
    };
    // set-up of every plan (workspace, preconditioner factors) on its batch stream
    each_plan(b, all, [&](size_t i) {
        rcs[i] = gmres_create(b->plans[i], freqs[i], nf[i], ports[i], np[i], opts, b->streams[i], &runs[i]);
        if (rcs[i]) msgs[i] = sie_last_error();
    });
    if (int rc = first_error("set-up")) { cleanup(); return rc; }
    std::vector<size_t> live(all);           // runs not finished
    std::vector<int64_t> launches(n, 0);
    while (!live.empty()) {
        std::vector<char> need(n, 0);
        each_plan(b, live, [&](size_t i) {
            bool nd = false;
            rcs[i] = gmres_top(runs[i], nd);
            need[i] = nd;
            if (rcs[i]) msgs[i] = sie_last_error();
        });
        if (int rc = first_error("residual")) { cleanup(); return rc; }
        std::vector<size_t> cyc;
        for (size_t i : live)
            if (need[i]) cyc.push_back(i);
        if (cyc.empty()) break;
        for (size_t i : cyc)
            if (int rc = gmres_begin(runs[i])) { cleanup(); return rc; }
        // the cycle's first step eagerly (it uploads each product's coefficients and
        // sets the kernels' attributes), then the running set's step as one graph
        for (size_t i : cyc)
            if (int rc = gmres_step(runs[i], false)) { cleanup(); return rc; }
        std::vector<size_t> running;
        for (size_t i : cyc) {
            SIE_CUDA(cudaStreamSynchronize(b->streams[i]));
            if (!gmres_stepped(runs[i])) running.push_back(i);
        }
        cudaGraphExec_t exec = nullptr;
        while (!running.empty()) {
            if (!exec) {
                if (int rc = capture_gmres_step(b, runs, running, launches, &exec)) { cleanup(); return rc; }
            }
            cudaError_t e = cudaGraphLaunch(exec, b->origin);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->origin);
            if (e != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                cleanup();
                return fail(SIE_ERR_CUDA, std::string("sie_batch_solve_graph: replay: ") + cudaGetErrorString(e));
            }
            ++b->replays;
            std::vector<size_t> still;
            for (size_t i : running) {
                b->plans[i]->launches += launches[i];
                if (!gmres_stepped(runs[i])) still.push_back(i);
            }
            if (still.size() != running.size()) {   // a cycle ended: capture the smaller set
                cudaGraphExecDestroy(exec);
                exec = nullptr;
            }
            running.swap(still);
        }
        if (exec) cudaGraphExecDestroy(exec);
        std::vector<char> cont(n, 0);
        each_plan(b, cyc, [&](size_t i) {
            bool c = false;
            rcs[i] = gmres_end(runs[i], c);
            cont[i] = c;
            if (rcs[i]) msgs[i] = sie_last_error();
        });
        if (int rc = first_error("cycle")) { cleanup(); return rc; }
        // a run leaves when its top needed no cycle (converged, capped or broken
        // down) or when its cycle end says the solve is over
        std::vector<size_t> next;
        for (size_t i : live)
            if (need[i] && cont[i]) next.push_back(i);
        live.swap(next);
    }
    int first_rc = SIE_OK;
    std::string first_msg;
    for (size_t i = 0; i < n; ++i) {
        const int rc = gmres_finish(runs[i], Z_out[i], st_out ? &st_out[i] : nullptr);
        runs[i] = nullptr;
        if (rc && !first_rc) {
            first_rc = rc;
            first_msg = "sie_batch_solve_graph: plan " + std::to_string(i) + ": " + sie_last_error();
        }
    }
    if (first_rc) return fail(first_rc, first_msg);
    return SIE_OK;
}
