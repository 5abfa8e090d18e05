// k_csr.cu -- Krylov passes for sparse systems in CSR form.
//
// SpMV.  w = A' (s_j V_j) with A' = [[A, b], [0, 0]] when the state carries the
// constant-1 variable (Sec. 2.1): row r < n gets sum_e val[e] x[col[e]] +
// b[r] x[n], row n is zero.  One thread per row; the row sum is a double in
// the FP64 form and an error-free float pair (Dot2) in the FP32 form.
//
// Arnoldi (Alg. 1) for general A, one iteration j per column as two passes
// over the stored basis V_0..V_j (each V_l stored unnormalised, read scale
// s_l):
//   dots:   h1_l = v_l . w and g_l = v_l . v_j for l <= j (one read of V)
//   update: w -= sum_l (h1_l + h2_l) v_l with h2 = h1 - G h1,
//           beta = ||w||, P[:, j+1] = C w / beta  (second read of V)
// G = V^T V is the Gram matrix of the basis, grown by one row per iteration
// from the g_l of the same pass.  h2 = V^T (w - V h1) evaluated through G is
// the second projection of classical Gram-Schmidt with reorthogonalisation
// (CGS2) without re-reading V for it; Alg. 1 uses modified Gram-Schmidt, which
// gives the same H and P in exact arithmetic.
//
// Lanczos (Alg. 3) for symmetric CSR: SpMV fused with alpha_j = v_j . A v_j,
// then w = A v_j - alpha_j v_j - beta_j v_{j-1} over three rotating buffers.
//
// All scalars stay on the device; the last block of each pass finishes the
// deterministic reduction and writes them.
#include <type_traits>

#include "kv_internal.h"
#include "reduce.cuh"

namespace kv {

constexpr int CNT = 256;           // threads per block
constexpr int CR = 8;              // rows per thread in the Gram-Schmidt passes
constexpr int CCHUNK = CNT * CR;   // rows per block

struct ArnoldiDev {  // per-column device scratch of the Arnoldi passes
    double g[KV_MAX_M + 1][KV_MAX_M + 1];  // Gram matrix of the stored basis (normalised)
    double c[KV_MAX_M + 1];                // update coefficients (h1 + h2) s_l
};

template <typename T>
struct VecArgs {
    T* base;       // column 0's (m+1) vectors of N; column c at base + c * cstride
    int64_t cstride;
};

// ------------------------------------------------------------------ SpMV --
template <typename T, bool ALPHA>
__global__ void __launch_bounds__(CNT) k_spmv(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                              const T* __restrict__ val, const double* __restrict__ b,
                                              VecArgs<T> V, int xslot, int wslot, int64_t n, int64_t N,
                                              const int* aug, ColState* st, double* H, int m, int j,
                                              double* partials, unsigned* counters, int64_t nbx) {
    const int cidx = blockIdx.y;
    ColState* s = st + cidx;
    if (s->done) return;
    const T* X = V.base + cidx * V.cstride + (int64_t)xslot * N;
    T* Wv = V.base + cidx * V.cstride + (int64_t)wslot * N;
    const double sj = s->s[j];
    const bool ag = aug[cidx] != 0;
    double acc_alpha = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * CNT + threadIdx.x; r < N; r += (int64_t)gridDim.x * CNT) {
        double y;
        if (r < n) {
            if constexpr (std::is_same<T, float>::value) {
                Dot2f d;
                for (int64_t e = rp[r]; e < rp[r + 1]; ++e) d.add_prod(val[e], X[col[e]]);
                y = d.value();
            } else {
                double d = 0.0;
                for (int64_t e = rp[r]; e < rp[r + 1]; ++e) d = fma(val[e], X[col[e]], d);
                y = d;
            }
            if (ag && b) y = fma(b[r], (double)X[n], y);
            y *= sj;
        } else {
            y = 0.0;  // the constant variable's row of A' is zero
        }
        const T yt = (T)y;
        Wv[r] = yt;
        if (ALPHA) acc_alpha = fma(sj * (double)X[r], (double)yt, acc_alpha);
    }
    if (!ALPHA) return;
    __shared__ double sh[CNT / 32];
    __shared__ int flag;
    const double part = block_sum<CNT>(acc_alpha, sh);
    if (!grid_arrive(part, partials + cidx * nbx, counters + cidx, blockIdx.x, gridDim.x, &flag)) return;
    const double tot = grid_finish<CNT>(partials + cidx * nbx, gridDim.x, counters + cidx, sh);
    if (threadIdx.x == 0) H[(int64_t)cidx * (m + 1) * m + (int64_t)j * m + j] = tot;  // alpha_j
}

// gather of C x by a whole block; result in thread 0
template <typename T>
__device__ double cgather(const CDesc& cd, int r, const T* x, double* sh) {
    double v = 0.0;
    for (int64_t e = cd.rp[r] + threadIdx.x; e < cd.rp[r + 1]; e += CNT) v += cd.val[e] * (double)__ldcg(x + cd.col[e]);
    return block_sum<CNT>(v, sh);
}

// Shared epilogue of every pass that produces w = unnormalised v_{j+1}:
// beta = ||w||, breakdown test against ||A v_j||^2 = sum_l H[l][j]^2 + beta^2,
// scale, H entries, P column.  Runs in the last block, all threads.
template <typename T>
__device__ void finish_vector(double nw2, const T* W, ColState* s, double* H, double* P, const CDesc& cd, int m,
                              int j, bool symmetric, double* sh) {
    __shared__ double snext;
    __shared__ int cont;
    if (threadIdx.x == 0) {
        const double beta = sqrt(nw2);
        H[(int64_t)(j + 1) * m + j] = beta;
        double nav2 = beta * beta;
        for (int l = 0; l <= j; ++l) nav2 += H[(int64_t)l * m + j] * H[(int64_t)l * m + j];
        if (!(beta > 1e-12 * sqrt(nav2)) || !isfinite(beta)) {
            s->done = 1;
            s->m_used = j + 1;
            cont = 0;
        } else {
            if (symmetric && j + 1 < m) H[(int64_t)j * m + (j + 1)] = beta;
            s->s[j + 1] = 1.0 / beta;
            snext = 1.0 / beta;
            cont = (j + 1 < m) ? 1 : 0;
        }
    }
    __syncthreads();
    if (!cont) return;
    for (int r = 0; r < cd.o; ++r) {
        const double v = cgather<T>(cd, r, W, sh);
        if (threadIdx.x == 0) P[(int64_t)r * m + (j + 1)] = snext * v;
    }
}

// ------------------------------------------------------ Lanczos update --
template <typename T, bool FIRST>
__global__ void __launch_bounds__(CNT) k_lanczos3_update(VecArgs<T> V, int wslot, int vslot, int pslot, int64_t N,
                                                         ColState* st, double* Hall, double* Pall, CDesc cd, int m,
                                                         int j, double* partials, unsigned* counters, int64_t nbx) {
    const int cidx = blockIdx.y;
    ColState* s = st + cidx;
    if (s->done) return;
    double* H = Hall + (int64_t)cidx * (m + 1) * m;
    T* Wv = V.base + cidx * V.cstride + (int64_t)wslot * N;
    const T* Vj = V.base + cidx * V.cstride + (int64_t)vslot * N;
    const T* Vp = V.base + cidx * V.cstride + (int64_t)pslot * N;
    const double alpha = H[(int64_t)j * m + j];
    const double ca = -alpha * s->s[j];
    const double cb = FIRST ? 0.0 : -H[(int64_t)j * m + (j - 1)] * s->s[j - 1];
    typename AccOf<T>::type acc;
    for (int64_t r = (int64_t)blockIdx.x * CNT + threadIdx.x; r < N; r += (int64_t)gridDim.x * CNT) {
        double w = fma(ca, (double)Vj[r], (double)Wv[r]);
        if (!FIRST) w = fma(cb, (double)Vp[r], w);
        const T wt = (T)w;
        Wv[r] = wt;
        acc.add_prod(wt, wt);
    }
    __shared__ double sh[CNT / 32];
    __shared__ int flag;
    const double part = block_sum<CNT>(acc.value(), sh);
    if (!grid_arrive(part, partials + cidx * nbx, counters + cidx, blockIdx.x, gridDim.x, &flag)) return;
    const double tot = grid_finish<CNT>(partials + cidx * nbx, gridDim.x, counters + cidx, sh);
    finish_vector<T>(tot, Wv, s, H, Pall + (int64_t)cidx * cd.o * m, cd, m, j, true, sh);
}

// --------------------------------------------------------- Arnoldi dots --
// partials layout: [column][q][block], q < 2 (j+1): h1 then g
template <typename T>
__global__ void __launch_bounds__(CNT) k_arnoldi_dots(VecArgs<T> V, int64_t N, ColState* st, double* Hall,
                                                      ArnoldiDev* ad, int m, int j, double* partials,
                                                      unsigned* counters, int64_t nbx) {
    const int cidx = blockIdx.y;
    ColState* s = st + cidx;
    if (s->done) return;
    const T* Vc = V.base + cidx * V.cstride;
    const T* W = Vc + (int64_t)(j + 1) * N;
    const T* Vj = Vc + (int64_t)j * N;
    __shared__ double wsum[2 * (KV_MAX_M + 1)][CNT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * CCHUNK + threadIdx.x;
    // FP64 form: double products; FP32 form: each thread's CR products summed
    // in float (one rounding per product and add), then one double add per
    // basis vector -- the FP64 pipe is 1/64 of the float pipe on this GPU
    T wv[CR], vv[CR];
#pragma unroll
    for (int k = 0; k < CR; ++k) {
        const int64_t r = r0 + (int64_t)k * CNT;
        wv[k] = r < N ? W[r] : (T)0;
        vv[k] = r < N ? Vj[r] : (T)0;
    }
    for (int l = 0; l <= j; ++l) {
        const T* Vl = Vc + (int64_t)l * N;
        T at = 0, gt = 0;
#pragma unroll
        for (int k = 0; k < CR; ++k) {
            const int64_t r = r0 + (int64_t)k * CNT;
            const T x = r < N ? Vl[r] : (T)0;
            at = fma(x, wv[k], at);
            gt = fma(x, vv[k], gt);
        }
        double a = (double)at, g = (double)gt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (lane == 0) {
            wsum[l][warp] = a;
            wsum[KV_MAX_M + 1 + l][warp] = g;
        }
    }
    __syncthreads();
    const int K = j + 1;
    double* part = partials + (int64_t)cidx * nbx * 2 * (KV_MAX_M + 1);
    for (int q = threadIdx.x; q < 2 * K; q += CNT) {
        const int row = q < K ? q : (KV_MAX_M + 1 + q - K);
        double v = 0.0;
        for (int w = 0; w < CNT / 32; ++w) v += wsum[row][w];
        part[(int64_t)q * nbx + blockIdx.x] = v;
    }
    __shared__ int flag;
    if (!block_ticket(counters + cidx, gridDim.x, &flag)) return;
    // last block: totals, scaled by the read scales
    __shared__ double tot[2 * (KV_MAX_M + 1)];
    for (int q = threadIdx.x; q < 2 * K; q += CNT) {
        double v = 0.0;
        for (int64_t bb = 0; bb < gridDim.x; ++bb) v += __ldcg(part + (int64_t)q * nbx + bb);
        const int l = q < K ? q : q - K;
        tot[q] = v * s->s[l] * (q < K ? 1.0 : s->s[j]);
    }
    if (threadIdx.x == 0) *(counters + cidx) = 0u;
    __syncthreads();
    ArnoldiDev* A = ad + cidx;
    double* H = Hall + (int64_t)cidx * (m + 1) * m;
    // Gram row j: g_l = v_l . v_j
    for (int l = threadIdx.x; l <= j; l += CNT) {
        A->g[j][l] = tot[K + l];
        A->g[l][j] = tot[K + l];
    }
    __syncthreads();
    // h2 = h1 - G h1 ; coefficient of v_l in the update is h1 + h2
    for (int l = threadIdx.x; l <= j; l += CNT) {
        double gh = 0.0;
        for (int k = 0; k <= j; ++k) gh = fma(A->g[l][k], tot[k], gh);
        const double h = tot[l] + (tot[l] - gh);
        H[(int64_t)l * m + j] = h;
        A->c[l] = h * s->s[l];
    }
}

// ------------------------------------------------------- Arnoldi update --
template <typename T>
__global__ void __launch_bounds__(CNT) k_arnoldi_update(VecArgs<T> V, int64_t N, ColState* st, double* Hall,
                                                        double* Pall, ArnoldiDev* ad, CDesc cd, int m, int j,
                                                        double* partials, unsigned* counters, int64_t nbx) {
    const int cidx = blockIdx.y;
    ColState* s = st + cidx;
    if (s->done) return;
    T* Vc = V.base + cidx * V.cstride;
    T* W = Vc + (int64_t)(j + 1) * N;
    const ArnoldiDev* A = ad + cidx;
    __shared__ double cf[KV_MAX_M + 1];
    for (int l = threadIdx.x; l <= j; l += CNT) cf[l] = A->c[l];
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * CCHUNK + threadIdx.x;
    T wv[CR];
#pragma unroll
    for (int k = 0; k < CR; ++k) {
        const int64_t r = r0 + (int64_t)k * CNT;
        wv[k] = r < N ? W[r] : (T)0;
    }
    for (int l = 0; l <= j; ++l) {
        const T* Vl = Vc + (int64_t)l * N;
        if constexpr (std::is_same<T, float>::value) {
            const CoefPair c = split_coef(-cf[l]);  // the coefficient to ~48 bits
#pragma unroll
            for (int k = 0; k < CR; ++k) {
                const int64_t r = r0 + (int64_t)k * CNT;
                if (r < N) {
                    const float v = Vl[r];
                    wv[k] = fmaf(c.hi, v, fmaf(c.lo, v, wv[k]));
                }
            }
        } else {
            const double c = cf[l];
#pragma unroll
            for (int k = 0; k < CR; ++k) {
                const int64_t r = r0 + (int64_t)k * CNT;
                if (r < N) wv[k] = fma(-c, Vl[r], wv[k]);
            }
        }
    }
    typename AccOf<T>::type acc;
#pragma unroll
    for (int k = 0; k < CR; ++k) {
        const int64_t r = r0 + (int64_t)k * CNT;
        if (r < N) {
            const T wt = (T)wv[k];
            W[r] = wt;
            acc.add_prod(wt, wt);
        }
    }
    __shared__ double sh[CNT / 32];
    __shared__ int flag;
    const double part = block_sum<CNT>(acc.value(), sh);
    if (!grid_arrive(part, partials + cidx * nbx, counters + cidx, blockIdx.x, gridDim.x, &flag)) return;
    const double tot = grid_finish<CNT>(partials + cidx * nbx, gridDim.x, counters + cidx, sh);
    finish_vector<T>(tot, W, s, Hall + (int64_t)cidx * (m + 1) * m, Pall + (int64_t)cidx * cd.o * m, cd, m, j,
                     false, sh);
}

// ------------------------------------------------------------ launchers --
static int64_t row_blocks(int64_t N) { return (N + CCHUNK - 1) / CCHUNK; }
static int64_t spmv_blocks(int64_t N) {
    int64_t b = (N + CNT - 1) / CNT;
    return b > 152 * 16 ? 152 * 16 : b;
}

int64_t csr_scratch_slots(int64_t N) {  // reduction partials per column
    const int64_t nb = row_blocks(N) > spmv_blocks(N) ? row_blocks(N) : spmv_blocks(N);
    return nb * 2 * (KV_MAX_M + 1);
}

size_t csr_arnoldi_dev_bytes() { return sizeof(ArnoldiDev); }

template <typename T>
static int run_csr_column_t(Prob* p, int j0, int ncols, void* V, ArnoldiDev* ad, bool lanczos) {
    const Sys* s = p->sys;
    const int64_t N = p->N, n = s->n;
    cudaStream_t st = p->ctx->stream;
    VecArgs<T> va{(T*)V, (int64_t)p->nvec * N};
    const int m = p->m;
    CDesc cd{p->o, p->d_crp, p->d_ccol, p->d_cval};
    ColState* stp = p->d_state + j0;
    double* H = p->d_H + (int64_t)j0 * (m + 1) * m;
    double* P = p->d_P + (int64_t)j0 * p->o * m;
    int* aug = p->d_aug + j0;
    const int64_t nbx = row_blocks(N) > spmv_blocks(N) ? row_blocks(N) : spmv_blocks(N);
    double* partials = p->red.partials;
    unsigned* counters = p->d_counters;
    dim3 gs((unsigned)spmv_blocks(N), (unsigned)ncols), gr((unsigned)row_blocks(N), (unsigned)ncols);
    for (int it = 0; it < m; ++it) {
        if (lanczos) {
            const int vs = it % 3, ws = (it + 1) % 3, ps = (it + 2) % 3;
            {
                LaunchScope ls(p->ctx, "csr_spmv");
                k_spmv<T, true><<<gs, CNT, 0, st>>>(s->d_rp, s->d_col, (const T*)s->d_val, s->d_b, va, vs, ws, n, N,
                                                   aug, stp, H, m, it, partials, counters, nbx);
                KV_CHECK_CUDA(cudaGetLastError());
            }
            LaunchScope ls(p->ctx, "csr_lanczos_update");
            if (it == 0)
                k_lanczos3_update<T, true><<<gs, CNT, 0, st>>>(va, ws, vs, ps, N, stp, H, P, cd, m, it, partials,
                                                              counters, nbx);
            else
                k_lanczos3_update<T, false><<<gs, CNT, 0, st>>>(va, ws, vs, ps, N, stp, H, P, cd, m, it, partials,
                                                               counters, nbx);
            KV_CHECK_CUDA(cudaGetLastError());
        } else {
            {
                LaunchScope ls(p->ctx, "csr_spmv");
                k_spmv<T, false><<<gs, CNT, 0, st>>>(s->d_rp, s->d_col, (const T*)s->d_val, s->d_b, va, it, it + 1, n,
                                                    N, aug, stp, H, m, it, partials, counters, nbx);
                KV_CHECK_CUDA(cudaGetLastError());
            }
            {
                LaunchScope ls(p->ctx, "arnoldi_dots");
                k_arnoldi_dots<T><<<gr, CNT, 0, st>>>(va, N, stp, H, ad, m, it, partials, counters, nbx);
                KV_CHECK_CUDA(cudaGetLastError());
            }
            LaunchScope ls(p->ctx, "arnoldi_update");
            k_arnoldi_update<T><<<gr, CNT, 0, st>>>(va, N, stp, H, P, ad, cd, m, it, partials, counters, nbx);
            KV_CHECK_CUDA(cudaGetLastError());
        }
    }
    return KV_OK;
}

// Runs the Krylov iterations of columns j0 .. j0+ncols-1 (all of the same
// method), whose initial vectors are already in slot 0 of their vector sets.
int launch_csr_columns(Prob* p, int j0, int ncols, void* V, bool lanczos) {
    ArnoldiDev* ad = (ArnoldiDev*)p->d_arnoldi + j0;
    if (p->prec == KV_FP32) return run_csr_column_t<float>(p, j0, ncols, V, ad, lanczos);
    return run_csr_column_t<double>(p, j0, ncols, V, ad, lanczos);
}

}  // namespace kv
