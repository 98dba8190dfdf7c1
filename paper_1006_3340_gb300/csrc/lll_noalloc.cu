// lll_noalloc.cu -- lll_simulate_noalloc: a simulation entry point that
// allocates no device memory.
//
// Who needs it: services that reserve all their device memory once at
// start-up (through their own pool) and forbid any later cudaMalloc, and
// latency-bound callers that cannot afford the device-wide synchronisation
// cudaMalloc / cudaFree may imply.  lll_simulate may grow its per-call
// scratch with cudaMalloc; this entry point never does.
//
// Its scratch (per-block path state and per-block payoff partials of the
// path kernel) lives in the file-scope array below: kScratchBytes on every
// GPU that loads the library, held until the process exits.  Host code must
// not use the array's name as a device address (on the host it names a
// stand-in object); the device address comes from cudaGetSymbolAddress.  It
// is looked up again on every call made outside a stream capture (after a
// cudaDeviceReset the module, and with it the array, may be reloaded at
// another address); a call made during a capture, when the lookup is not
// allowed, uses the address the last uncaptured call found on that device.
#include <cstdio>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/lll.h"
#include "lll_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20; // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
// capturing: the caller's stream is being captured, so only the address an
// earlier uncaptured call found may be used (cudaErrorStreamCaptureUnsupported
// if there is none).
cudaError_t scratch_address(int device, bool capturing, void **out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!capturing) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = ptr;
    }
    if (!g_scratch_addr[device]) return cudaErrorStreamCaptureUnsupported;
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

size_t round256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

extern "C" int lll_simulate_noalloc(lll_ctx *ctx, int scheme, uint64_t first_path, uint64_t paths,
                                    uint64_t seed, double *d_sums)
{
    using namespace lll;
    if (!ctx) return record_error(nullptr, LLL_EINVAL, "ctx is NULL");
    if (!d_sums) return record_error(ctx, LLL_EINVAL, "d_sums is NULL");
    LaunchPlan plan;
    int rc = plan_launch(ctx, scheme, first_path, paths, seed, &plan);
    if (rc != LLL_OK) return rc;
    const size_t state_bytes = round256(sizeof(float) * plan.state_floats_per_block * plan.grid);
    const size_t need = state_bytes + sizeof(double) * plan.partial_doubles_per_block * plan.grid;
    if (need > kScratchBytes) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "lll_simulate_noalloc needs %zu bytes of scratch for this launch (%d blocks); "
                      "its static maximum is %zu bytes",
                      need, plan.grid, kScratchBytes);
        return record_error(ctx, LLL_EUNSUPPORTED, msg);
    }
    int current = -1;
    cudaError_t e = cudaGetDevice(&current);
    if (e != cudaSuccess || current != plan.device)
        return record_error(ctx, LLL_ECUDA, "the context's device must be current");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(plan.stream, &cap);
    const bool capturing = e != cudaSuccess || cap != cudaStreamCaptureStatusNone;
    if (e != cudaSuccess) cudaGetLastError(); // keep the launch check below from seeing this query's error
    void *base = nullptr;
    e = scratch_address(current, capturing, &base);
    if (e == cudaErrorStreamCaptureUnsupported)
        return record_error(ctx, LLL_ESTATE,
                            "lll_simulate_noalloc: make one call outside stream capture first on this device");
    if (e != cudaSuccess) {
        std::string msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return record_error(ctx, LLL_ECUDA, msg.c_str());
    }
    // Nothing here has to start at zero: the kernel zeroes each path's state
    // when it starts the path, and every block of the grid writes all of its
    // partials before the final reduction reads them.
    PathArgs a = plan.args;
    a.state = static_cast<float *>(base);
    a.partials = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + state_bytes);
    e = (cudaError_t)launch_plan(plan, a);
    if (e != cudaSuccess) {
        std::string msg = std::string("path kernel launch: ") + cudaGetErrorString(e);
        return record_error(ctx, LLL_ECUDA, msg.c_str());
    }
    e = (cudaError_t)launch_finalize(a.partials, plan.grid, plan.n_out, d_sums, plan.stream);
    if (e != cudaSuccess) {
        std::string msg = std::string("finalize launch: ") + cudaGetErrorString(e);
        return record_error(ctx, LLL_ECUDA, msg.c_str());
    }
    return LLL_OK;
}
