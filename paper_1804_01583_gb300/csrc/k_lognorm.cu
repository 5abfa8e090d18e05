// k_lognorm.cu -- upper bound of the largest eigenvalue of (A + A^T)/2 for a
// CSR matrix, the e^{max(mu,0) T} factor of the a-posteriori bound of
// Lemma 1 (Sec. 4.2; the lemma's nu(B) for B = -A is -mu(A)).
//
// The same pass returns max_i sum_j |a'_ij| (rounded up), for a symmetric A
// a bound of ||A||_2 that sizes the squarings of the Lanczos exponentials.
//
// Gershgorin on the symmetric part: every eigenvalue of (A + A^T)/2 lies in a
// disc around a_ii of radius sum_{j != i} |a_ij + a_ji| / 2, so
//   mu <= max_i  a_ii + (sum_{j != i} |a_ij| + sum_{j != i} |a_ji|) / 2,
// and for A' = [[A, b], [0, 0]] row i gains |b_i|/2 and the extra row is
// sum_i |b_i| / 2.
//
// Column sums need a scatter.  To keep the result the same on every run, each
// |a_ij| is rounded up to a fixed-point grid (2^-36 of the largest off-diagonal
// magnitude) and the sums are exact 64-bit integer atomics, which do not
// depend on their order; rounding up, and directed rounding in the final
// combination, keep the result an upper bound.  The maximum over rows is an
// atomicMax on an order-preserving integer image of the doubles.
#include <math.h>

#include "kv_internal.h"

namespace kv {

constexpr int LNT = 256;
constexpr double FIX_SCALE = 68719476736.0;  // 2^36

__device__ __forceinline__ unsigned long long order_key(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

static double from_order_key(unsigned long long k) {
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k;
    double x;
    memcpy(&x, &b, sizeof(x));
    return x;
}

struct LnScratch {
    unsigned long long amax_bits, bmax_bits;  // non-negative doubles: raw bits order like values
    unsigned long long g_key, ga_key;         // order keys of max_i g_i and max_i g'_i
    unsigned long long bsum;                  // fixed-point sum of |b_i| / bmax
    unsigned long long rsum_bits;             // max_i sum_j |a'_ij| (non-negative double bits)
};

template <typename T>
__global__ void __launch_bounds__(LNT) k_ln_max(const int64_t* rp, const int32_t* col, const T* val, const double* b,
                                                int64_t n, LnScratch* sc) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (LNT / 32);
    double am = 0.0, bm = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * (LNT / 32) + (threadIdx.x >> 5); r < n; r += warps) {
        for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32)
            if (col[e] != r) am = fmax(am, fabs((double)val[e]));
        if (b && lane == 0) bm = fmax(bm, fabs(b[r]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
        bm = fmax(bm, __shfl_xor_sync(0xffffffffu, bm, o));
    }
    if (lane == 0) {
        atomicMax(&sc->amax_bits, (unsigned long long)__double_as_longlong(am));
        atomicMax(&sc->bmax_bits, (unsigned long long)__double_as_longlong(bm));
    }
}

template <typename T>
__global__ void __launch_bounds__(LNT) k_ln_colsum(const int64_t* rp, const int32_t* col, const T* val, const double* b,
                                                   int64_t n, LnScratch* sc, unsigned long long* csum) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (LNT / 32);
    const double amax = __longlong_as_double((long long)sc->amax_bits);
    const double bmax = __longlong_as_double((long long)sc->bmax_bits);
    for (int64_t r = (int64_t)blockIdx.x * (LNT / 32) + (threadIdx.x >> 5); r < n; r += warps) {
        if (amax > 0.0)
            for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
                if (col[e] == r) continue;
                const double q = ceil(__dmul_ru(fabs((double)val[e]) / amax, FIX_SCALE));
                atomicAdd(&csum[col[e]], (unsigned long long)q);
            }
        if (b && lane == 0 && bmax > 0.0)
            atomicAdd(&sc->bsum, (unsigned long long)ceil(__dmul_ru(fabs(b[r]) / bmax, FIX_SCALE)));
    }
}

template <typename T>
__global__ void __launch_bounds__(LNT) k_ln_rows(const int64_t* rp, const int32_t* col, const T* val, const double* b,
                                                 int64_t n, LnScratch* sc, const unsigned long long* csum) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (LNT / 32);
    const double amax = __longlong_as_double((long long)sc->amax_bits);
    unsigned long long gk = 0ULL, gak = 0ULL;
    double rmax = 0.0;  // the largest absolute row sum, rounded up
    for (int64_t r = (int64_t)blockIdx.x * (LNT / 32) + (threadIdx.x >> 5); r < n; r += warps) {
        double d = 0.0, off = 0.0;
        for (int64_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
            const double v = (double)val[e];
            if (col[e] == r) d = v;
            else off = __dadd_ru(off, fabs(v));
        }
        for (int o = 16; o > 0; o >>= 1) {
            off = __dadd_ru(off, __shfl_xor_sync(0xffffffffu, off, o));
            d += __shfl_xor_sync(0xffffffffu, d, o);  // one lane holds the diagonal, the others 0
        }
        if (lane == 0) {
            const double cs = __dmul_ru(__dmul_ru((double)csum[r], amax), 1.0 / FIX_SCALE);
            const double g = __dadd_ru(d, __dmul_ru(0.5, __dadd_ru(off, cs)));
            gk = max(gk, order_key(g));
            if (b) gak = max(gak, order_key(__dadd_ru(g, __dmul_ru(0.5, fabs(b[r])))));
            rmax = fmax(rmax, __dadd_ru(__dadd_ru(fabs(d), off), b ? fabs(b[r]) : 0.0));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        gk = max(gk, __shfl_xor_sync(0xffffffffu, gk, o));
        gak = max(gak, __shfl_xor_sync(0xffffffffu, gak, o));
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    if (lane == 0) {
        atomicMax(&sc->g_key, gk);
        if (b) atomicMax(&sc->ga_key, gak);
        atomicMax(&sc->rsum_bits, (unsigned long long)__double_as_longlong(rmax));
    }
}

int csr_lognorm_bounds(Sys* s, const double* b_host, double* mu, double* mu_aug, double* row_abs_max) {
    Ctx* c = s->ctx;
    LnScratch* sc = (LnScratch*)c->arena.alloc(sizeof(LnScratch));
    unsigned long long* csum = (unsigned long long*)c->arena.alloc((size_t)s->n * sizeof(unsigned long long));
    if (!sc || !csum) {
        c->arena.free(sc);
        c->arena.free(csum);
        set_error("kv_system_csr: pool cannot hold the log-norm scratch");
        return KV_ENOMEM;
    }
    cudaStream_t st = c->stream;
    const double* db = b_host ? s->d_b : nullptr;
    int64_t blocks = (s->n + (LNT / 32) - 1) / (LNT / 32);
    if (blocks > 152 * 16) blocks = 152 * 16;
    cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(LnScratch), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(csum, 0, (size_t)s->n * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        if (s->val_prec == KV_FP32) {
            const float* v = (const float*)s->d_val;
            k_ln_max<float><<<(unsigned)blocks, LNT, 0, st>>>(s->d_rp, s->d_col, v, db, s->n, sc);
            k_ln_colsum<float><<<(unsigned)blocks, LNT, 0, st>>>(s->d_rp, s->d_col, v, db, s->n, sc, csum);
            k_ln_rows<float><<<(unsigned)blocks, LNT, 0, st>>>(s->d_rp, s->d_col, v, db, s->n, sc, csum);
        } else {
            const double* v = (const double*)s->d_val;
            k_ln_max<double><<<(unsigned)blocks, LNT, 0, st>>>(s->d_rp, s->d_col, v, db, s->n, sc);
            k_ln_colsum<double><<<(unsigned)blocks, LNT, 0, st>>>(s->d_rp, s->d_col, v, db, s->n, sc, csum);
            k_ln_rows<double><<<(unsigned)blocks, LNT, 0, st>>>(s->d_rp, s->d_col, v, db, s->n, sc, csum);
        }
        e = cudaGetLastError();
    }
    LnScratch h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    c->arena.free(sc);
    c->arena.free(csum);
    if (e != cudaSuccess) {
        set_error("kv_system_csr: log-norm bound failed: %s", cudaGetErrorString(e));
        return KV_ECUDA;
    }
    *mu = from_order_key(h.g_key);
    *mu_aug = *mu;
    memcpy(row_abs_max, &h.rsum_bits, sizeof(double));
    if (b_host) {
        double bmax;
        memcpy(&bmax, &h.bmax_bits, sizeof(bmax));
        // the constant row of A': sum_i |b_i| / 2, rounded up
        const double brow = nextafter(0.5 * (double)h.bsum * bmax / FIX_SCALE * (1.0 + 4e-16), INFINITY);
        *mu_aug = std::max(from_order_key(h.ga_key), brow);
    }
    return KV_OK;
}

}  // namespace kv
