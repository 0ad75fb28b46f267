// Polynomial products for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a product:
// hosts that own all device memory through their own allocator or a fixed
// budget reserved at start-up (a library must not take memory behind their
// back), and latency-critical loops where an allocation's implicit
// device-wide synchronisation, or the chance that it fails part-way through a
// run, is unacceptable.  polymul_mod_p_batch_static() serves them: it is
// polymul_mod_p_batch() with the fused schedule, except that the scratch
// space of the larger transforms is a fixed array in this file instead of a
// caller workspace.
//
// The array is a file-scope __device__ variable of kStaticScratchBytes; every
// GPU that loads the library holds it until the process exits.  Host code
// cannot use the symbol's name as a device address (it names a host-side
// stand-in), so the first call on each device, with that device current,
// looks the address up with cudaGetSymbolAddress and caches it together with
// the id of the context it belongs to.  That first call should therefore
// come before any stream capture.  A call from a different context of the
// same device (after cudaDeviceReset, say) looks the address up again.
// All calls share the one array and it keeps the last call's contents: calls
// whose work overlaps on the GPU (on different streams, or from several host
// threads) race on it and must be serialised by the caller.  No word of the
// scratch needs to start at zero: each call writes every scratch word it
// later reads.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/gbntt.h"
#include "kernels.h"
#include "plan.h"
#include "tma.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // context of each cached address

// Device address of g_static_scratch on the current device: looked up on
// the first call per device and again whenever the current context is not
// the one the cached address came from.
int scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long ctx = gbntt::current_context_id();
    if (!g_scratch_addr[device] || ctx == 0 || ctx != g_scratch_ctx[device]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            gbntt_set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return NTT_ERR_CUDA;
        }
        g_scratch_addr[device] = ptr;
        g_scratch_ctx[device] = gbntt::current_context_id();   // the look-up makes the context current
    }
    *out = g_scratch_addr[device];
    return NTT_OK;
}

}  // namespace

extern "C" int polymul_mod_p_batch_static(const ntt_plan* plan, const void* d_a, size_t na,
                                          const void* d_b, size_t nb, size_t batch, void* d_c,
                                          void* stream) {
    if (!plan) return NTT_ERR_ARG;
    if (batch == 0) return NTT_OK;
    const size_t need = gbntt::polymul_ws_bytes(plan, batch, NTT_SCHED_FUSED);
    if (need > kStaticScratchBytes) {
        gbntt_set_error("polymul_mod_p_batch_static: " + std::to_string(batch) +
                        " products need " + std::to_string(need) +
                        " bytes of scratch; the fixed array holds " +
                        std::to_string(kStaticScratchBytes) + " (use fewer products per call)");
        return NTT_ERR_WORKSPACE;
    }
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return NTT_ERR_CUDA;
    }
    if (device < 0 || device >= kMaxDevices || device != plan->device) {
        gbntt_set_error("polymul_mod_p_batch_static: the plan's device must be current");
        return NTT_ERR_ARG;
    }
    // set-up on every device's first call, whether or not this product
    // needs scratch, so that later calls never look anything up
    void* scratch = nullptr;
    const int rc = scratch_address(device, &scratch);
    if (rc != NTT_OK) return rc;
    return polymul_mod_p_batch(plan, d_a, na, d_b, nb, batch, d_c, NTT_SCHED_FUSED, scratch,
                               kStaticScratchBytes, stream);
}
