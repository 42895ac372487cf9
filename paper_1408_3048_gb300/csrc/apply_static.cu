// y = A x without any device allocation at call time.
//
// mm_apply_A computes A x = P^T [N^-1 [P x]] through a time-domain intermediate (one
// value per sample) that lives in a buffer the plan allocated.  This variant runs the
// same two kernels (Toeplitz with fused de-pointing, then the pixel scatter) but keeps
// that intermediate in a fixed array compiled into the library, so the call itself
// never asks the CUDA runtime for memory.  It is meant for callers that must not
// allocate once they are running: code whose device memory is already handed out to a
// pool it does not control (a framework's caching allocator that reserved the GPU), or
// code on a latency-critical path where a cudaMalloc could fail or stall the device.
//
// The array lives in each device's memory from the module's load until the process
// exits.  Its device address is looked up by mm_plan (static_scratch_setup, with the
// plan's device current), which also makes the CUDA runtime load this module and create
// the array then, not inside a call.  The array is shared by every call in the process:
// every call overwrites all the entries it reads (every sample of every interval is
// written by the Toeplitz kernel before the scatter reads it), so nothing needs
// clearing; but calls whose work overlaps on the GPU -- on two streams, or from two host
// threads -- race on the array.
#include <mutex>

#include "mm_internal.h"

namespace mm {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_tod[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

struct StaticCall {
    mm_plan_t plan;
    int precision;
    const void* x;
    void* y;
};

void static_apply(void* ctx) {
    const StaticCall& c = *static_cast<const StaticCall*>(ctx);
    if (c.plan == nullptr) throw Error{MM_ERR_ARG, "null plan"};
    Plan* P = reinterpret_cast<Plan*>(c.plan);
    if (c.x == nullptr || c.y == nullptr) throw Error{MM_ERR_ARG, "null vector"};
    if (c.precision != MM_FP64 && c.precision != MM_FP32)
        throw Error{MM_ERR_ARG, "precision must be MM_FP64 or MM_FP32"};
    const size_t need = (size_t)P->nt * (c.precision == MM_FP64 ? 8 : 4);
    if (need > kStaticScratchBytes)
        throw Error{MM_ERR_ARG, "mm_apply_A_static: nt = " + std::to_string(P->nt) + " needs " +
                                    std::to_string(need) + " bytes of time-domain scratch, above the static limit of " +
                                    std::to_string(kStaticScratchBytes) + " bytes (use mm_apply_A)"};
    void* scratch = static_scratch_ptr(P->device);
    if (c.precision == MM_FP64) {
        launch_toeplitz<double>(*P, P->tz64, nullptr, static_cast<const double*>(c.x), static_cast<double*>(scratch),
                                nullptr, P->stream);
        launch_scatter<double>(*P, static_cast<const double*>(scratch), static_cast<double*>(c.y), nullptr,
                               P->stream);
    } else {
        launch_toeplitz<float>(*P, P->tz32, nullptr, static_cast<const float*>(c.x), static_cast<float*>(scratch),
                               nullptr, P->stream);
        launch_scatter<float>(*P, static_cast<const float*>(scratch), static_cast<float*>(c.y), nullptr, P->stream);
    }
    check_cuda(cudaStreamSynchronize(P->stream), "stream synchronize");
}

}  // namespace

// With `device` current: the device address of g_static_tod on it (re-read for every new
// plan, so a device reset between plans cannot leave a stale address behind).
void static_scratch_setup(int device) {
    if (device < 0 || device >= kMaxDevices) throw Error{MM_ERR_ARG, "device index beyond the static scratch table"};
    void* p = nullptr;
    check_cuda(cudaGetSymbolAddress(&p, g_static_tod), "cudaGetSymbolAddress(static scratch)");
    std::lock_guard<std::mutex> lock(g_static_mu);
    g_static_addr[device] = p;
}

void* static_scratch_ptr(int device) {
    if (device < 0 || device >= kMaxDevices) throw Error{MM_ERR_ARG, "device index beyond the static scratch table"};
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (g_static_addr[device] == nullptr) throw Error{MM_ERR_STATE, "static scratch not set up on this device"};
    return g_static_addr[device];
}

size_t static_scratch_bytes() { return kStaticScratchBytes; }

}  // namespace mm

extern "C" mm_status mm_apply_A_static(mm_plan_t plan, int precision, const void* x, void* y) {
    mm::StaticCall c{plan, precision, x, y};
    return mm::run_guarded(reinterpret_cast<mm::Plan*>(plan), mm::static_apply, &c);
}
