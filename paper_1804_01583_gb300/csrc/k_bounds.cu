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

// Many columns (the transpose dynamics make i large cheap): the sums over
// the columns are split into chunks, one thread per (chunk, row, step), and
// the chunks are added in order by k_bounds_reduce.
constexpr int BCHUNK_MIN = 1024;

static int bounds_chunk(int ncol) {
    int c = BCHUNK_MIN;
    while ((ncol + c - 1) / c > 65535) c *= 2;
    return c;
}

__global__ void k_bounds_partial(const double* __restrict__ basis, int ncol, int o, int steps, const double* zlo,
                                 const double* zhi, int chunk, double* part) {
    const int64_t S = steps + 1;
    const int64_t total = (int64_t)o * S;
    const int64_t e = (int64_t)blockIdx.x * BNT + threadIdx.x;
    if (e >= total) return;
    const int r = (int)(e / S);
    const int k = (int)(e - (int64_t)r * S);
    const int j0 = blockIdx.y * chunk, j1 = min(ncol, j0 + chunk);
    double l = 0.0, h = 0.0;
    for (int j = j0; j < j1; ++j) {
        const double p = basis[((int64_t)j * o + r) * S + k];
        const double a = p * zlo[j], c = p * zhi[j];
        l += a < c ? a : c;
        h += a < c ? c : a;
    }
    part[((int64_t)blockIdx.y * 2) * total + e] = l;
    part[((int64_t)blockIdx.y * 2 + 1) * total + e] = h;
}

__global__ void k_bounds_reduce(const double* __restrict__ part, int nchunks, int o, int steps, const double* theta,
                                double* lo, double* hi, int* key) {
    const int64_t S = steps + 1;
    const int64_t total = (int64_t)o * S;
    for (int64_t e = (int64_t)blockIdx.x * BNT + threadIdx.x; e < total; e += (int64_t)gridDim.x * BNT) {
        double l = 0.0, h = 0.0;
        for (int q = 0; q < nchunks; ++q) {
            l += part[((int64_t)q * 2) * total + e];
            h += part[((int64_t)q * 2 + 1) * total + e];
        }
        lo[e] = l;
        hi[e] = h;
        const int r = (int)(e / S);
        if (h >= theta[r]) atomicMin(key, (int)(e - (int64_t)r * S) * o + r);
    }
}

size_t bounds_scratch_doubles(int ncol, int o, int steps) {
    if (ncol <= BCHUNK_MIN) return 0;
    const int64_t nch = (ncol + bounds_chunk(ncol) - 1) / bounds_chunk(ncol);
    return (size_t)nch * 2 * o * (steps + 1);
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
    if (p->i <= BCHUNK_MIN) {
        LaunchScope ls(p->ctx, "bounds");
        k_bounds<<<(unsigned)(g < 1 ? 1 : g), BNT, 0, s>>>(p->d_basis, p->i, p->o, p->steps, p->d_zlo, p->d_zhi,
                                                       p->d_theta, p->d_lo, p->d_hi, p->d_viol);
        KV_CHECK_CUDA(cudaGetLastError());
    } else {
        LaunchScope ls(p->ctx, "bounds");
        const int chunk = bounds_chunk(p->i);
        const int nch = (p->i + chunk - 1) / chunk;
        const dim3 gp((unsigned)((total + BNT - 1) / BNT), (unsigned)nch);
        k_bounds_partial<<<gp, BNT, 0, s>>>(p->d_basis, p->i, p->o, p->steps, p->d_zlo, p->d_zhi, chunk,
                                            p->d_bpart);
        k_bounds_reduce<<<(unsigned)(g < 1 ? 1 : g), BNT, 0, s>>>(p->d_bpart, nch, p->o, p->steps, p->d_theta,
                                                                p->d_lo, p->d_hi, p->d_viol);
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
