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
// The array is shared by every call in the process (on each device it lives in that
// device's memory from module load until exit).  Every call overwrites all the entries
// it reads (every sample of every interval is written by the Toeplitz kernel before the
// scatter reads it), so nothing needs clearing; but calls whose work overlaps on the
// GPU -- on two streams, or from two host threads -- race on the array.
#include <mutex>

#include "mm_internal.h"

namespace mm {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_tod[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};

// Device address of g_static_tod on the current device (looked up once per device).
void* static_scratch() {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) throw Error{MM_ERR_ARG, "device index beyond the static scratch table"};
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (g_static_addr[dev] == nullptr) {
        void* p = nullptr;
        check_cuda(cudaGetSymbolAddress(&p, g_static_tod), "cudaGetSymbolAddress(static scratch)");
        g_static_addr[dev] = p;
    }
    return g_static_addr[dev];
}

}  // namespace
}  // namespace mm

extern "C" mm_status mm_apply_A_static(mm_plan_t plan, int precision, const void* x, void* y) {
    using namespace mm;
    if (plan == nullptr) return MM_ERR_ARG;
    Plan* P = reinterpret_cast<Plan*>(plan);
    try {
        if (x == nullptr || y == nullptr) throw Error{MM_ERR_ARG, "null vector"};
        if (precision != MM_FP64 && precision != MM_FP32)
            throw Error{MM_ERR_ARG, "precision must be MM_FP64 or MM_FP32"};
        const size_t need = (size_t)P->nt * (precision == MM_FP64 ? 8 : 4);
        if (need > kStaticScratchBytes)
            throw Error{MM_ERR_ARG, "mm_apply_A_static: nt = " + std::to_string(P->nt) +
                                        " needs " + std::to_string(need) + " bytes of time-domain scratch, above "
                                        "the static limit of " + std::to_string(kStaticScratchBytes) +
                                        " bytes (use mm_apply_A)"};
        void* scratch = static_scratch();
        if (precision == MM_FP64) {
            launch_toeplitz<double>(*P, P->tz64, nullptr, static_cast<const double*>(x),
                                    static_cast<double*>(scratch), nullptr, P->stream);
            launch_scatter<double>(*P, static_cast<const double*>(scratch), static_cast<double*>(y), nullptr,
                                   P->stream);
        } else {
            launch_toeplitz<float>(*P, P->tz32, nullptr, static_cast<const float*>(x),
                                   static_cast<float*>(scratch), nullptr, P->stream);
            launch_scatter<float>(*P, static_cast<const float*>(scratch), static_cast<float*>(y), nullptr,
                                  P->stream);
        }
        check_cuda(cudaStreamSynchronize(P->stream), "stream synchronize");
        return MM_OK;
    } catch (const Error& e) {
        P->err = e.msg;
        return e.st;
    }
}
