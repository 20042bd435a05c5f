// Allocation-free variant of the even-odd Schur operator.
//
// plq_schur_apply needs an odd-parity half field for the intermediate
// H_oe * in, which its caller allocates.  Some callers cannot allocate device
// memory at the time they apply the operator: code that hands all device
// memory to its own pool or allocator and forbids others from calling
// cudaMalloc, real-time loops that must not take the allocator's locks or
// risk its latency, and callers held to a device-memory budget fixed at
// start-up.  plq_schur_apply_noalloc keeps that intermediate in a fixed
// device array that is part of the library image instead, so the call itself
// allocates nothing.
#include <cuda.h>

#include <mutex>

#include "plq_internal.cuh"

namespace plq {
namespace {

constexpr size_t kScratchBytes = PLQ_NOALLOC_SCRATCH_BYTES;

// The intermediate odd half field of plq_schur_apply_noalloc.  It lives in
// every GPU that loads the library until the process exits, and all calls on
// a device share it.
static __device__ __align__(256) unsigned char schur_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
struct ScratchAddr {
    void *ptr = nullptr;
    unsigned long long ctx_id = 0;  // driver context the address belongs to
};
ScratchAddr g_scratch[kMaxDevices];

// Identity of the driver context current in this thread.  The module holding
// schur_scratch is loaded once per context, and cudaDeviceReset destroys the
// primary context (and the module with it); context ids are never reused in a
// process, so a changed id means the cached address is stale.  The two driver
// calls are taken through the runtime's entry-point query, so the library
// needs no link against the driver library.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

plq_status current_context_id(unsigned long long *id) {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void **>(&g_ctx_get_current),
                                                         12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void **>(&g_ctx_get_id), 12000,
                                                 cudaEnableDefault, &q2);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetDriverEntryPointByVersion");
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !g_ctx_get_current ||
            !g_ctx_get_id) {
            g_ctx_get_current = nullptr;
            g_ctx_get_id = nullptr;
            return set_error(PLQ_ERR_CUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not available");
        }
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return set_error(PLQ_ERR_CUDA, "no current CUDA context");
    if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return set_error(PLQ_ERR_CUDA, "cuCtxGetId failed");
    return PLQ_OK;
}

// Device address of schur_scratch on `device` (which must be current).  In
// host code the symbol itself is only a host-side stand-in, so the address is
// looked up on the first call in a context of the device and cached with that
// context's id.
plq_status scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return set_error(PLQ_ERR_ARG, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_mutex);
    unsigned long long id = 0;
    PLQ_TRY(current_context_id(&id));
    ScratchAddr &c = g_scratch[device];
    if (!c.ptr || c.ctx_id != id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, schur_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(schur_scratch)");
        c.ptr = p;
        c.ctx_id = id;
    }
    *out = c.ptr;
    return PLQ_OK;
}

}  // namespace
}  // namespace plq

using namespace plq;

extern "C" plq_status plq_schur_apply_noalloc(plq_ctx *c, void *out, const void *in, double kappa, int dagger,
                                              int prec, void *stream) {
    if (!c) return set_error(PLQ_ERR_ARG, "null context");
    auto aligned = [](const void *p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (!aligned(out) || !aligned(in)) return set_error(PLQ_ERR_ARG, "null or misaligned field pointer");
    if (out == in) return set_error(PLQ_ERR_ARG, "in and out must be distinct");
    if (!valid_prec(prec)) return set_error(PLQ_ERR_ARG, "bad precision %d", prec);
    const size_t need = spinor_site_bytes(prec) * (size_t)c->lat.Vh;
    if (need > kScratchBytes)
        return set_error(PLQ_ERR_ARG,
                         "plq_schur_apply_noalloc: the odd half field needs %zu bytes, above the fixed scratch of "
                         "%zu bytes (use plq_schur_apply with a caller-owned tmp)",
                         need, kScratchBytes);
    if (!c->gauge[prec].ptr) return set_error(PLQ_ERR_STATE, "no gauge field uploaded for precision %d", prec);
    PLQ_CUDA(cudaSetDevice(c->device));
    void *tmp = nullptr;
    PLQ_TRY(scratch_address(c->device, &tmp));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // tmp = H_oe in: every element of the used part of the scratch is written
    // here before it is read below, so nothing left by an earlier call leaks in.
    // Both launches take the context's tuned configuration, as plq_schur_apply.
    HopArgs a;
    a.in = in;
    a.out = tmp;
    a.gauge = c->gauge[prec].ptr;
    a.gblock = c->gauge[prec].block;
    a.out_parity = 1;
    a.lat = c->lat;
    apply_tune(c, prec, 1, a);
    a.dagger = dagger ? 1 : 0;
    PLQ_TRY(launch_hop(a, prec, c->gauge[prec].reals, EPI_PLAIN, s));
    // out = in - kappa^2 H_eo tmp
    HopArgs b;
    b.in = tmp;
    b.out = out;
    b.gauge = c->gauge[prec].ptr;
    b.gblock = c->gauge[prec].block;
    b.out_parity = 0;
    b.lat = c->lat;
    apply_tune(c, prec, 1, b);
    b.dagger = dagger ? 1 : 0;
    b.x = in;
    b.a = -kappa * kappa;
    return launch_hop(b, prec, c->gauge[prec].reals, EPI_XPAY, s);
}
