// reduce.cuh -- deterministic reductions and error-free float accumulation.
//
// A grid reduction writes one double per block to `partials`, then the block
// that arrives last (ticket on `counter`) sums all partials in a fixed order
// (thread t adds slots t, t+NT, ... in sequence, then a fixed tree), so the
// result does not depend on block scheduling and repeats bit for bit.  No
// floating-point atomics are used.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kv {

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) sh[t >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (t < 32) {
        r = (t < NT / 32) ? sh[t] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// Writes this block's partial and reports whether this block is the last to
// finish.  Every thread of the block must call it.  `slot` is the block's
// linear index, `nblocks` the grid size.
__device__ __forceinline__ bool grid_arrive(double partial, double* partials, unsigned* counter,
                                            int64_t slot, int64_t nblocks, int* sh_flag) {
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    if (t == 0) {
        partials[slot] = partial;
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        *sh_flag = (ticket == (unsigned)(nblocks - 1)) ? 1 : 0;
    }
    __syncthreads();
    const bool last = *sh_flag != 0;
    if (last) __threadfence();
    return last;
}

// Ticket for passes whose partials were written by several threads of the
// block: every thread fences its own writes before the block takes a ticket.
// Every thread must call it; returns true in the last block to arrive.
__device__ __forceinline__ bool block_ticket(unsigned* counter, int64_t nblocks, int* sh_flag) {
    __threadfence();
    __syncthreads();
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    if (t == 0) {
        const unsigned ticket = atomicAdd(counter, 1u);
        *sh_flag = (ticket == (unsigned)(nblocks - 1)) ? 1 : 0;
    }
    __syncthreads();
    const bool last = *sh_flag != 0;
    if (last) __threadfence();
    return last;
}

// Fixed-order sum of n partials by the (last) block; result in thread 0.
// Resets the counter for the next reduction.
template <int NT>
__device__ __forceinline__ double grid_finish(const double* partials, int64_t n, unsigned* counter,
                                              double* sh) {
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    double v = 0.0;
    for (int64_t i = t; i < n; i += NT) v += __ldcg(partials + i);
    const double r = block_sum<NT>(v, sh);
    if (t == 0) *counter = 0u;
    return r;
}

// ---------------------------------------------------------------------------
// Error-free accumulation in float pairs (Ogita, Rump, Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 26(6), 2005: TwoSum / TwoProduct /
// Dot2).  The _rn intrinsics keep the compiler from contracting the
// transformations into fused operations, which would break them.
struct Dot2f {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);     // a*b = p + pe exactly
        const float t = __fadd_rn(s, p);
        const float z = __fadd_rn(t, -s);
        const float e = __fadd_rn(__fadd_rn(s, -__fadd_rn(t, -z)), __fadd_rn(p, -z));  // s+p = t+e exactly
        s = t;
        c = __fadd_rn(c, __fadd_rn(e, pe));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

struct Dot2d {  // plain double accumulation for the FP64 form
    double s = 0.0;
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

// A double coefficient as an unevaluated float pair hi + lo (about 48 bits).
struct CoefPair {
    float hi, lo;
};
__host__ __device__ __forceinline__ CoefPair split_coef(double c) {
    const float h = (float)c;
    return CoefPair{h, (float)(c - (double)h)};
}

template <typename T>
struct AccOf;
template <>
struct AccOf<double> {
    using type = Dot2d;
};
template <>
struct AccOf<float> {
    using type = Dot2f;
};

}  // namespace kv
