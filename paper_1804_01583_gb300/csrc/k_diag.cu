// k_diag.cu -- the device's FP64 instruction rate, measured.
//
// The FP64 grid iteration is bound by the FP64 pipe, not by HBM, so its
// roofline needs the rate at which this device retires FP64 fused
// multiply-adds and additions.  Each thread runs eight independent
// dependency chains of FP64_RATE_ITERS operations; the grid is eight blocks
// of 256 threads per SM (enough warps to keep the pipe busy); the rate is
// operations per second over the best of five timed launches (CUDA events
// on a stream of its own, after one untimed launch).
#include "kv_internal.h"

namespace kv {

constexpr int FP64_RATE_ITERS = 4096;
constexpr int FP64_RATE_NT = 256;

__global__ void __launch_bounds__(FP64_RATE_NT) k_fp64_fma_rate(double* out, double a, double b) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = 1e-3 * threadIdx.x + i;
    for (int it = 0; it < FP64_RATE_ITERS; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(FP64_RATE_NT) k_fp64_add_rate(double* out, double a) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = 1e-3 * threadIdx.x + i;
    for (int it = 0; it < FP64_RATE_ITERS; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = x[i] + a;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace kv

extern "C" int kv_diag_fp64_rate(int device, double* fma_per_s, double* add_per_s) {
    using namespace kv;
    if (!fma_per_s || !add_per_s) {
        set_error("kv_diag_fp64_rate: NULL argument");
        return KV_EINVAL;
    }
    DeviceGuard dg(device);
    if (dg.err != cudaSuccess) {
        set_error("kv_diag_fp64_rate: device %d", device);
        return KV_EINVAL;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) {
        set_error("kv_diag_fp64_rate: multiprocessor count of device %d", device);
        return KV_ECUDA;
    }
    const int blocks = 8 * sms;
    const double threads = (double)blocks * FP64_RATE_NT;
    double* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best[2] = {1e30f, 1e30f};
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * (size_t)blocks * FP64_RATE_NT);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
        for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, st);
            if (kind == 0) k_fp64_fma_rate<<<blocks, FP64_RATE_NT, 0, st>>>(out, 0.999, 1e-3);
            else k_fp64_add_rate<<<blocks, FP64_RATE_NT, 0, st>>>(out, 1e-3);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0 && ms < best[kind]) best[kind] = ms;  // rep 0: warm-up
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        set_error("kv_diag_fp64_rate: %s", cudaGetErrorString(e));
        return KV_ECUDA;
    }
    const double ops = 8.0 * FP64_RATE_ITERS * threads;
    *fma_per_s = ops / (best[0] * 1e-3);
    *add_per_s = ops / (best[1] * 1e-3);
    return KV_OK;
}
