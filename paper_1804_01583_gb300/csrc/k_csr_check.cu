// k_csr_check.cu -- device side of kv_system_csr: the column checks and the
// FP32 rounding of the values, on the uploaded arrays.
//
// The column indices are checked where they already are after the upload (or
// where the caller keeps them, for device arrays): every index must lie in
// [0, n) and increase strictly within its row.  One warp takes a row, its lanes
// the row's entries; the smallest offending entry index is kept with an
// atomicMin, which is the entry a sequential scan in storage order reports
// first.  Row pointers are checked on the host before this runs (they bound
// every read here and size the allocations).
//
// FP32 storage: the doubles are uploaded through a staging buffer and rounded
// to nearest-even on the device (__double2float_rn), the rounding of a host
// (float) cast, so the stored values are the same bits either way.
#include "kv_internal.h"

namespace kv {

constexpr int CKT = 256;

__global__ void __launch_bounds__(CKT) k_csr_check_cols(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                        int64_t n, unsigned long long* first_bad) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (CKT / 32);
    unsigned long long bad = ~0ULL;
    for (int64_t r = (int64_t)blockIdx.x * (CKT / 32) + (threadIdx.x >> 5); r < n; r += warps) {
        const int64_t e0 = rp[r], e1 = rp[r + 1];
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t c = col[e];
            const bool out = c < 0 || (int64_t)c >= n;
            const bool order = e > e0 && c <= col[e - 1];
            if ((out || order) && (unsigned long long)e < bad) bad = (unsigned long long)e;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, bad, o);
        bad = x < bad ? x : bad;
    }
    if (lane == 0 && bad != ~0ULL) atomicMin(first_bad, bad);
}

__global__ void __launch_bounds__(CKT) k_round_to_float(const double* __restrict__ src, float* __restrict__ dst,
                                                        int64_t cnt) {
    const int64_t stride = (int64_t)gridDim.x * CKT;
    for (int64_t q = (int64_t)blockIdx.x * CKT + threadIdx.x; q < cnt; q += stride) dst[q] = __double2float_rn(src[q]);
}

static unsigned grid_for(int64_t work) {
    const int64_t g = (work + CKT - 1) / CKT;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

cudaError_t csr_check_cols_async(const int64_t* d_rp, const int32_t* d_col, int64_t n, unsigned long long* d_first_bad,
                                 cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d_first_bad, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_csr_check_cols<<<grid_for(n * 32), CKT, 0, st>>>(d_rp, d_col, n, d_first_bad);
    return cudaGetLastError();
}

cudaError_t round_to_float_async(const double* src, float* dst, int64_t cnt, cudaStream_t st) {
    if (cnt <= 0) return cudaSuccess;
    k_round_to_float<<<grid_for(cnt), CKT, 0, st>>>(src, dst, cnt);
    return cudaGetLastError();
}

}  // namespace kv
