// Launch profiling (diagnostic) and the integer-pipe throughput probe.
//
// Between ntt_profile_begin() and ntt_profile_end() every library launcher
// records a CUDA event on its own stream after each kernel it enqueues, so
// the interval between consecutive events is that kernel's device time on
// the stream it ran on.  Process-wide state; meant for one benchmarking
// thread.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/gbntt.h"
#include "kernels.h"
#include "plan.h"

namespace gbntt {

namespace {
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<const char*> names;   // names[i] ends at event i+1
    int used = 0;                     // events recorded
};
Prof g_prof;

cudaEvent_t next_event() {
    if (g_prof.used == static_cast<int>(g_prof.pool.size())) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g_prof.pool.push_back(e);
    }
    return g_prof.pool[g_prof.used++];
}
}  // namespace

void prof_mark(cudaStream_t st, const char* name) {
    if (!g_prof.on) return;
    if (g_prof.used == 0) {
        cudaEvent_t e0 = next_event();
        if (!e0) return;
        // the first interval starts at the first kernel's enqueue point
        cudaEventRecord(e0, st);
    }
    cudaEvent_t e = next_event();
    if (!e) return;
    cudaEventRecord(e, st);
    g_prof.names.push_back(name);
}

void prof_begin_call(cudaStream_t st) {
    if (!g_prof.on) return;
    if (g_prof.used == 0) {
        cudaEvent_t e0 = next_event();
        if (e0) cudaEventRecord(e0, st);
    } else {
        // a new call: restart the interval at this point so host gaps between
        // calls are not charged to the next kernel
        cudaEvent_t e = next_event();
        if (e) cudaEventRecord(e, st);
        g_prof.names.push_back(nullptr);
    }
}

// Integer throughput probe, 64 operations per thread per iteration on
// independent chains, every result feeding a store:
//   kind 0  32-bit multiply-adds (the multiply-add pipe);
//   kind 1  add and xor alternating along each chain (the ALU pipe);
//   kind 2  both at once, 1:1 -- eight multiply-add chains interleaved with
//           eight add/xor chains, so that each pipe has independent work
//           whenever the other is busy: the issue ceiling when integer work
//           splits evenly between the two pipes;
//   kind 3  32 x 32 -> 64-bit multiply-adds into 64-bit accumulators.
#define GB_MAD(x) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(m), "r"(c))
#define GB_ADD(x) asm volatile("add.u32 %0, %0, %1;" : "+r"(x) : "r"(m))
#define GB_XOR(x) asm volatile("xor.b32 %0, %0, %1;" : "+r"(x) : "r"(c))
#define GB_WIDE(x) asm volatile("{\n .reg .u32 lo;\n cvt.u32.u64 lo, %0;\n mad.wide.u32 %0, lo, %1, %0;\n}" \
                                : "+l"(x) : "r"(m))
#define GB_8(OP, a) OP(a##0); OP(a##1); OP(a##2); OP(a##3); OP(a##4); OP(a##5); OP(a##6); OP(a##7)

__global__ void k_int_probe(uint32_t* out, int iters, int kind, uint32_t seed) {
    uint32_t a0 = threadIdx.x ^ seed, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    uint32_t a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    uint32_t b0 = a0 ^ 0x55u, b1 = b0 + 1, b2 = b0 + 2, b3 = b0 + 3;
    uint32_t b4 = b0 + 4, b5 = b0 + 5, b6 = b0 + 6, b7 = b0 + 7;
    const uint32_t m = seed | 1u, c = seed >> 3;
    if (kind == 0) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 8; ++u) { GB_8(GB_MAD, a); }
        }
    } else if (kind == 1) {
        // add and xor alternate along each chain so no two consecutive
        // operations can merge into one three-input instruction
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                GB_8(GB_ADD, a);
                GB_8(GB_XOR, a);
            }
        }
    } else if (kind == 2) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                GB_8(GB_MAD, a);
                GB_8(GB_ADD, b);
                GB_8(GB_MAD, a);
                GB_8(GB_XOR, b);
            }
        }
    } else {
        uint64_t w0 = a0, w1 = a1, w2 = a2, w3 = a3, w4 = a4, w5 = a5, w6 = a6, w7 = a7;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 8; ++u) { GB_8(GB_WIDE, w); }
        }
        a0 = static_cast<uint32_t>(w0 ^ w1 ^ w2 ^ w3 ^ (w4 >> 32) ^ (w5 >> 32) ^ (w6 >> 32) ^ (w7 >> 32));
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7 ^
                                                 b0 ^ b1 ^ b2 ^ b3 ^ b4 ^ b5 ^ b6 ^ b7;
}

#undef GB_8
#undef GB_WIDE
#undef GB_XOR
#undef GB_ADD
#undef GB_MAD

}  // namespace gbntt

using namespace gbntt;

extern "C" int ntt_profile_begin(void) {
    g_prof.on = true;
    g_prof.used = 0;
    g_prof.names.clear();
    return NTT_OK;
}

extern "C" int ntt_profile_end(int max_kernels, float* ms_out, const char** names_out, int* count) {
    if (!count) return NTT_ERR_ARG;
    g_prof.on = false;
    int k = 0;
    if (g_prof.used > 0) {
        if (cudaEventSynchronize(g_prof.pool[g_prof.used - 1]) != cudaSuccess) {
            gbntt_set_error(cudaGetErrorString(cudaGetLastError()));
            return NTT_ERR_CUDA;
        }
        for (size_t i = 0; i < g_prof.names.size(); ++i) {
            if (!g_prof.names[i]) continue;     // a gap between calls
            if (k < max_kernels && ms_out && names_out) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, g_prof.pool[i], g_prof.pool[i + 1]);
                ms_out[k] = ms;
                names_out[k] = g_prof.names[i];
            }
            ++k;
        }
    }
    *count = k;
    g_prof.used = 0;
    g_prof.names.clear();
    return NTT_OK;
}

extern "C" int ntt_int_probe(unsigned kind, int blocks, int threads, int iters, void* stream,
                             double* ops_per_s) {
    if (!ops_per_s || blocks <= 0 || threads <= 0 || iters <= 0 || kind > 3) return NTT_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t* out = nullptr;
    if (cudaMalloc(&out, sizeof(uint32_t) * static_cast<size_t>(blocks) * threads) != cudaSuccess)
        return NTT_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_int_probe<<<blocks, threads, 0, st>>>(out, iters, static_cast<int>(kind), 12345u);   // warm-up
    cudaEventRecord(e0, st);
    k_int_probe<<<blocks, threads, 0, st>>>(out, iters, static_cast<int>(kind), 777u);
    cudaEventRecord(e1, st);
    int rc = NTT_OK;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
        gbntt_set_error(cudaGetErrorString(cudaGetLastError()));
        rc = NTT_ERR_CUDA;
    } else {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double ops = 64.0 * iters * static_cast<double>(blocks) * threads;
        *ops_per_s = ops / (ms * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
