// pfft_convolve_noalloc: the grid convolution of pfft_convolve without any
// device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// convolution: code running under a strict memory budget that was fixed at
// start-up, a real-time loop where cudaMalloc's implicit device
// synchronisation and unbounded latency are not acceptable, or a host
// framework that owns the allocator and forbids allocation outside its own
// pool.  pfft_convolve may grow the plan's scratch on first use of a batch
// size; this entry point never does.  Its only scratch is the file-scope device
// array below, which every GPU that loads the library holds until the process
// exits.
#include <mutex>

#include <cudaTypedefs.h>

#include "sie_plan.h"

using namespace sie;

namespace {

// Scratch for the convolution: one grid transformed along x, [2N_x][N_y][N_z]
// per grid, complex128 or complex64.  4 MiB holds one 128 x 64 x 32 grid in
// FP32 (the mixed form's convolution precision).
constexpr size_t kNoallocScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};   // unique id of the context the address belongs to

// Unique id of the current device's context (cuCtxGetId, reached through the
// runtime so that the library needs no link to the driver library), or 0 when
// the driver cannot say.  A device reset retires the primary context and the
// next runtime call creates a new one, with a new id, into which the module and
// its array may load at another address.
unsigned long long current_context_id() {
    using GetCurrent = PFN_cuCtxGetCurrent_v4000;
    using GetId = PFN_cuCtxGetId_v12000;
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f1);
            get_id = reinterpret_cast<GetId>(f2);
        }
        (void)cudaGetLastError();
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current device's context.  In
// host code the array's name is only a host-side stand-in, so the address is
// looked up with cudaGetSymbolAddress (with that device current) the first time
// a device is used and kept; it is looked up again when the device's context
// has changed since (after cudaDeviceReset), or on every call if the context's
// id cannot be read.
int scratch_address(void **out) {
    int dev = 0;
    SIE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SIE_ERR_ARG, "pfft_convolve_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(SIE_ERR_CUDA, std::string("pfft_convolve_noalloc: cudaGetSymbolAddress failed: ") +
                                          cudaGetErrorString(e));
        g_scratch_addr[dev] = ptr;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return SIE_OK;
}

}  // namespace

extern "C" int pfft_convolve_noalloc(pfft_plan *p, void *grid, int32_t nbatch, int32_t prec, void *cuda_stream) {
    if (!p || !grid || nbatch < 1) return fail(SIE_ERR_ARG, "pfft_convolve_noalloc: bad argument");
    if (prec != SIE_PREC_FP64 && prec != SIE_PREC_MIXED)
        return fail(SIE_ERR_ARG, "pfft_convolve_noalloc: bad precision");
    const size_t cb = prec == SIE_PREC_FP64 ? 16 : 8;
    // per grid: the x-transformed copy, and for planes larger than one CTA its y transform
    const size_t spec_bytes = size_t(p->Mx) * (p->Ny + (p->large_plane ? p->My : 0)) * p->Nz * cb;
    if (spec_bytes > kNoallocScratchBytes)
        return fail(SIE_ERR_ARG, "pfft_convolve_noalloc: one grid's transformed copies need " + std::to_string(spec_bytes) +
                                     " bytes, more than the fixed scratch of " +
                                     std::to_string(kNoallocScratchBytes) + " bytes; use pfft_convolve");
    (void)cudaGetLastError();
    void *spec = nullptr;
    int rc = scratch_address(&spec);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int32_t per_call = int32_t(kNoallocScratchBytes / spec_bytes);
    const size_t grid_bytes = size_t(p->Ng) * cb;
    // the forward pass writes every spectrum element the later passes read, so
    // nothing in the scratch has to be cleared between calls
    for (int32_t b = 0; b < nbatch; b += per_call) {
        const int32_t n = std::min(per_call, nbatch - b);
        rc = fft_conv_n(p, static_cast<char *>(grid) + size_t(b) * grid_bytes, spec, n, prec, s);
        if (rc) return rc;
    }
    SIE_CUDA(cudaStreamSynchronize(s));
    return SIE_OK;
}
