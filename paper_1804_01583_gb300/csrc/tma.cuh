// tma.cuh -- mbarrier and TMA tile-load helpers shared by the single-pass grid
// kernels (k_stencil_tma.cu: FP32 storage, k_stencil_tma64.cu: FP64), and the
// host-side tensor-map encoder they use.
//
// Every wait is bounded: mbar_wait polls at most `limit` times and reports
// failure instead of spinning forever; the kernels act on a failed wait by
// setting the column's status word and draining their own copies.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kv {

constexpr long WAIT_LIMIT = 1L << 22;

__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, long limit = WAIT_LIMIT) {
    for (long it = 0; it < limit; ++it)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}
// One tiled 3-D TMA load into shared memory, completion counted in bytes on
// the mbarrier.  The x coordinate times the element size must be a multiple
// of 16 bytes (callers keep x a multiple of 4 floats or 2 doubles).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(saddr(dst)),
        "l"((uint64_t)map), "r"(saddr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// hi + lo += x with the rounding error of the float add kept in lo (TwoSum,
// Knuth; six float operations, valid for any ordering of |hi| and |x|).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// Host: cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link against libcuda); nullptr when the driver does not provide it.
typedef CUresult (*PfnEncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
PfnEncodeTiled tensor_map_encoder();

// A 3-D tiled map over an nx x ny x nz grid vector (x fastest) of 4- or
// 8-byte elements with a box_w x box_h x 1 box; coordinates outside the grid
// read as zero.  Returns KV_OK or KV_ECUDA (message set).
int make_grid_map(CUtensorMap* m, void* base, int64_t nx, int64_t ny, int64_t nz, int elem_bytes, int box_w,
                  int box_h);

}  // namespace kv
