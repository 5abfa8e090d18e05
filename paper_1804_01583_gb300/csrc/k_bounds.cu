// k_bounds.cu -- per-step output interval over the box initial set, first
// violation of y_r >= theta_r and the counter-example vertex.
//
// The per-step LP of Sec. 2.1 (two copies of the variables, the basis matrix
// between them, the initial and unsafe constraints) has, for a box z_j in
// [zlo_j, zhi_j] and a single half-space per output row, the closed-form
// optimum hi_r(k) = sum_j max(p zlo_j, p zhi_j) with p = basis[j][r][k]; the
// row is violated iff hi_r(k) >= theta_r, and the maximising vertex
// (z_j = zhi_j if p > 0, zlo_j if p < 0, midpoint if p == 0) is the
// counter-example initial point (Sec. 2, "a counter-example ... defined by an
// initial state x0 and time t").  Steps k = 0..steps are all checked.
#include <limits.h>

#include "kv_internal.h"

namespace kv {

constexpr int BNT = 256;
constexpr int KEY_NONE = 0x7f7f7f7f;  // cudaMemset(0x7f) pattern

__global__ void k_bounds(const double* __restrict__ basis, int ncol, int o, int steps, const double* zlo,
                         const double* zhi, const double* theta, double* lo, double* hi, int* key) {
    const int64_t S = steps + 1;
    const int64_t total = (int64_t)o * S;
    for (int64_t e = (int64_t)blockIdx.x * BNT + threadIdx.x; e < total; e += (int64_t)gridDim.x * BNT) {
        const int r = (int)(e / S);
        const int k = (int)(e - (int64_t)r * S);
        double l = 0.0, h = 0.0;
        for (int j = 0; j < ncol; ++j) {
            const double p = basis[((int64_t)j * o + r) * S + k];
            const double a = p * zlo[j], c = p * zhi[j];
            l += a < c ? a : c;
            h += a < c ? c : a;
        }
        lo[e] = l;
        hi[e] = h;
        if (h >= theta[r]) atomicMin(key, k * o + r);  // smallest step, then smallest row
    }
}

__global__ void k_bounds_finish(const double* __restrict__ basis, int ncol, int o, int steps, const double* zlo,
                                const double* zhi, const double* hi, const int* key, double* zstar,
                                double* ystar) {
    const int kk = *key;
    if (kk == KEY_NONE) return;
    const int64_t S = steps + 1;
    const int k = kk / o, r = kk - (kk / o) * o;
    for (int j = threadIdx.x; j < ncol; j += BNT) {
        const double p = basis[((int64_t)j * o + r) * S + k];
        zstar[j] = p > 0 ? zhi[j] : (p < 0 ? zlo[j] : 0.5 * (zlo[j] + zhi[j]));
    }
    if (threadIdx.x == 0) *ystar = hi[(int64_t)r * S + k];
}

int launch_bounds(Prob* p) {
    cudaStream_t s = p->ctx->stream;
    KV_CHECK_CUDA(cudaMemsetAsync(p->d_viol, 0x7f, sizeof(int), s));
    const int64_t total = (int64_t)p->o * (p->steps + 1);
    int64_t g = (total + BNT - 1) / BNT;
    if (g > 152 * 4) g = 152 * 4;
    {
        LaunchScope ls(p->ctx, "bounds");
        k_bounds<<<(unsigned)(g < 1 ? 1 : g), BNT, 0, s>>>(p->d_basis, p->i, p->o, p->steps, p->d_zlo, p->d_zhi,
                                                       p->d_theta, p->d_lo, p->d_hi, p->d_viol);
        KV_CHECK_CUDA(cudaGetLastError());
    }
    {
        LaunchScope ls(p->ctx, "bounds_finish");
        k_bounds_finish<<<1, BNT, 0, s>>>(p->d_basis, p->i, p->o, p->steps, p->d_zlo, p->d_zhi, p->d_hi, p->d_viol,
                                          p->d_zstar, p->d_ystar);
        KV_CHECK_CUDA(cudaGetLastError());
    }
    return KV_OK;
}

}  // namespace kv
