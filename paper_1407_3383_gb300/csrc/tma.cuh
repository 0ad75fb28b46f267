// Tensor-memory-accelerator (TMA) loads for the transform kernels: one
// cp.async.bulk.tensor copy brings a whole tile of an operand into shared
// memory, completed on an mbarrier, instead of one strided load per word per
// thread.  Every wait is bounded: on timeout a block sets the library's
// device error flag (read by ntt_device_status()), waits once more (bounded)
// for its copy, and returns.
#pragma once
#include <cuda.h>   // CUtensorMap (types only; the encoder is reached through the runtime)
#include <cstdint>

namespace gbntt {

// Bit set in the library's device error flag (a pointer every TMA kernel
// receives) by a block whose bounded wait ran out.
constexpr int kDevErrTmaTimeout = 1;
constexpr long kMbarSpinLimit = 1L << 24;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Wait for phase `parity` of the barrier, at most `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long limit) {
    const unsigned a = smem_u32(bar);
    for (long it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 3-D tiled load of the box at (x, y, z) into shared memory, completing
// `bytes` transactions on `bar`.  x * element size must be a multiple of 16.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// One block-wide TMA load of `bytes` into dst, waited for by every thread.
// Returns false (after flagging the error and a second bounded wait) when
// the copy did not complete in time; the whole block then sees false.
__device__ __forceinline__ bool tma_block_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                                  unsigned bytes, uint64_t* bar, int* err) {
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, bytes);
        tma_load_3d(dst, map, x, y, z, bar);
    }
    const bool ok = mbar_wait(bar, 0, kMbarSpinLimit);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(err, kDevErrTmaTimeout);
        mbar_wait(bar, 0, kMbarSpinLimit);
        return false;
    }
    return true;
}

// Host: encode a 3-D tiled tensor map (row-major, dims[0] fastest; strides
// in bytes for dims 1 and 2).  Returns false when the encoder is unavailable
// or rejects the layout (the caller then takes the plain-load kernels).
bool encode_tensor_map_3d(CUtensorMap* map, CUtensorMapDataType type, void* base, const uint64_t dims[3],
                          const uint64_t strides_bytes[2], const uint32_t box[3]);

// Host: the device address of the error flag on the current device.
int* device_error_flag();

// Host: a process-unique id of the calling thread's current CUDA context
// (cuCtxGetId), 0 when no context is current.  Addresses of __device__
// variables belong to one context: a cache of them keyed by this id is
// refreshed after a device reset creates a new one.
unsigned long long current_context_id();

}  // namespace gbntt
