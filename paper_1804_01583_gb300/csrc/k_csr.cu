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
#include <stdio.h>
#include <stdlib.h>

#include <string>
#include <type_traits>

#include "kv_internal.h"
#include "reduce.cuh"

namespace kv {

constexpr int CNT = 256;           // threads per block
// rows per thread in the dots pass (the FP32 form reduces each basis
// vector's per-thread partials across the warp as float pairs, so it needs
// no FP64 instruction per vector and can keep the rows per thread small)
template <typename T>
struct RowsPer {
    static constexpr int v = 8;
};
template <>
struct RowsPer<float> {
    static constexpr int v = 16;
};

// a + b = s + e exactly (TwoSum, Knuth), in float; the _rn intrinsics keep the
// compiler from contracting or reassociating it
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// butterfly sum over the warp of x as a float pair (hi, lo): every lane ends
// with the total, exact up to the float rounding of lo
__device__ __forceinline__ void warp_sum_pair(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        float sum, err;
        two_sum_f(hi, oh, sum, err);
        hi = sum;
        lo = __fadd_rn(__fadd_rn(lo, ol), err);
    }
}
constexpr int CCHUNK_MIN = CNT * 8;  // smallest rows per block (sizes the partials)

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

// ------------------------------------------------------------------ SpMM --
// W_c = s_c A' X_c for a group of G columns of a run (blockIdx.y = group):
// each row's values and column indices are read once for the G columns, and
// LPR lanes share a row (consecutive entries, combined by shuffles).  The
// group size and lanes per row are chosen per system by the autotuner.
template <typename T, int G, int LPR>
__global__ void __launch_bounds__(CNT) k_spmm(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                              const T* __restrict__ val, const double* __restrict__ b, VecArgs<T> V,
                                              int xslot, int wslot, int64_t n, int64_t N, const int* aug,
                                              const ColState* st, int j, int ncols) {
    const int cg0 = blockIdx.y * G;
    // the group's columns: X_k = xbase + k * cstride, W_k likewise
    const T* xbase = V.base + (int64_t)cg0 * V.cstride + (int64_t)xslot * N;
    T* wbase = V.base + (int64_t)cg0 * V.cstride + (int64_t)wslot * N;
    double sc[G];
    bool act[G], ag[G];
    int64_t off[G];  // inactive slots (past the run, or broken down) read the group's first column
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const int c = cg0 + k;
        act[k] = c < ncols && !st[c].done;
        sc[k] = act[k] ? st[c].s[j] : 0.0;
        ag[k] = act[k] && aug[c] != 0;
        off[k] = act[k] ? (int64_t)k * V.cstride : 0;
    }
    const int lane = threadIdx.x & 31, sub = lane % LPR;
    constexpr int WR = 32 / LPR;  // rows per warp per step
    const int64_t gw = ((int64_t)blockIdx.x * CNT + threadIdx.x) >> 5;
    const int64_t nw = (int64_t)gridDim.x * (CNT / 32);
    // warp-uniform loop: every lane reaches every shuffle
    for (int64_t rb = gw * WR; rb < N; rb += nw * WR) {
        const int64_t r = rb + lane / LPR;
        const bool inrow = r < n;
        const int64_t e0 = inrow ? rp[r] : 0, e1 = inrow ? rp[r + 1] : 0;
        if constexpr (std::is_same<T, float>::value) {
            Dot2f d[G];
            for (int64_t e = e0 + sub; e < e1; e += LPR) {
                const float v = val[e];
                const int c = col[e];
#pragma unroll
                for (int k = 0; k < G; ++k) d[k].add_prod(v, xbase[off[k] + c]);
            }
#pragma unroll
            for (int k = 0; k < G; ++k) {
#pragma unroll
                for (int o = LPR / 2; o > 0; o >>= 1) {  // error-free combination of lane pairs
                    const float s2 = __shfl_down_sync(0xffffffffu, d[k].s, o, LPR);
                    const float c2 = __shfl_down_sync(0xffffffffu, d[k].c, o, LPR);
                    const float t = __fadd_rn(d[k].s, s2);
                    const float z = __fadd_rn(t, -d[k].s);
                    const float err = __fadd_rn(__fadd_rn(d[k].s, -__fadd_rn(t, -z)), __fadd_rn(s2, -z));
                    d[k].s = t;
                    d[k].c = __fadd_rn(__fadd_rn(d[k].c, c2), err);
                }
            }
            if (sub == 0 && r < N) {
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    if (!act[k]) continue;
                    double y = 0.0;  // row n of A' (constant variable) is zero
                    if (inrow) {
                        y = d[k].value();
                        if (ag[k] && b) y = fma(b[r], (double)xbase[off[k] + n], y);
                    }
                    wbase[k * V.cstride + r] = (T)(sc[k] * y);
                }
            }
        } else {
            double d[G];
#pragma unroll
            for (int k = 0; k < G; ++k) d[k] = 0.0;
            for (int64_t e = e0 + sub; e < e1; e += LPR) {
                const double v = val[e];
                const int c = col[e];
#pragma unroll
                for (int k = 0; k < G; ++k) d[k] = fma(v, xbase[off[k] + c], d[k]);
            }
#pragma unroll
            for (int k = 0; k < G; ++k)
#pragma unroll
                for (int o = LPR / 2; o > 0; o >>= 1) d[k] += __shfl_down_sync(0xffffffffu, d[k], o, LPR);
            if (sub == 0 && r < N) {
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    if (!act[k]) continue;
                    double y = 0.0;
                    if (inrow) {
                        y = d[k];
                        if (ag[k] && b) y = fma(b[r], (double)xbase[off[k] + n], y);
                    }
                    wbase[k * V.cstride + r] = (T)(sc[k] * y);
                }
            }
        }
    }
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
    if (!cont || cd.o > PROJ_INLINE_MAX) return;  // launch_project takes many rows
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
    // per (basis vector, warp): the warp's sums as a double (FP64 form) or a
    // float pair (FP32 form), combined per block after the loop
    __shared__ double wsum[2 * (KV_MAX_M + 1)][CNT / 32];
    __shared__ float2 wsumf[2 * (KV_MAX_M + 1)][CNT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int CR = RowsPer<T>::v;
    const int64_t r0 = (int64_t)blockIdx.x * (CNT * CR) + threadIdx.x;
    T wv[CR], vv[CR], xa[CR], xb[CR];
#pragma unroll
    for (int k = 0; k < CR; ++k) {
        const int64_t r = r0 + (int64_t)k * CNT;
        wv[k] = r < N ? W[r] : (T)0;
        vv[k] = r < N ? Vj[r] : (T)0;
    }
    auto load = [&](T (&x)[CR], int l) {
        const T* Vl = Vc + (int64_t)l * N;
#pragma unroll
        for (int k = 0; k < CR; ++k) {
            const int64_t r = r0 + (int64_t)k * CNT;
            x[k] = r < N ? Vl[r] : (T)0;
        }
    };
    // this thread's products with basis vector l, reduced over the warp
    auto dots = [&](const T (&x)[CR], int l) {
        T at = 0, gt = 0;
#pragma unroll
        for (int k = 0; k < CR; ++k) {
            at = fma(x[k], wv[k], at);
            gt = fma(x[k], vv[k], gt);
        }
        if constexpr (std::is_same<T, float>::value) {
            float ah = at, al = 0.f, gh = gt, gl = 0.f;
            warp_sum_pair(ah, al);
            warp_sum_pair(gh, gl);
            if (lane == 0) {
                wsumf[l][warp] = make_float2(ah, al);
                wsumf[KV_MAX_M + 1 + l][warp] = make_float2(gh, gl);
            }
        } else {
            double a = at, g = gt;
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
    };
    // two register buffers: the loads of vector l+1 are in flight while the
    // products of vector l are formed and reduced
    load(xa, 0);
    for (int l = 0; l <= j; l += 2) {
        if (l + 1 <= j) load(xb, l + 1);
        dots(xa, l);
        if (l + 1 > j) break;
        if (l + 2 <= j) load(xa, l + 2);
        dots(xb, l + 1);
    }
    __syncthreads();
    const int K = j + 1;
    double* part = partials + (int64_t)cidx * nbx * 2 * (m + 1);
    for (int q = threadIdx.x; q < 2 * K; q += CNT) {
        const int row = q < K ? q : (KV_MAX_M + 1 + q - K);
        double v = 0.0;
        for (int w = 0; w < CNT / 32; ++w) {
            if constexpr (std::is_same<T, float>::value) v += (double)wsumf[row][w].x + (double)wsumf[row][w].y;
            else v += wsum[row][w];
        }
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
    // coefficients: double (FP64 form), or split once per block into float
    // pairs hi + lo carrying ~48 bits (FP32 form)
    __shared__ double cf[KV_MAX_M + 1];
    __shared__ float cfh[KV_MAX_M + 1], cfl[KV_MAX_M + 1];
    for (int l = threadIdx.x; l <= j; l += CNT) {
        cf[l] = A->c[l];
        const CoefPair c = split_coef(-A->c[l]);
        cfh[l] = c.hi;
        cfl[l] = c.lo;
    }
    __syncthreads();
    constexpr int CR = 8;  // no per-vector reduction here: short rows keep occupancy
    const int64_t r0 = (int64_t)blockIdx.x * (CNT * CR) + threadIdx.x;
    T wv[CR], xa[CR], xb[CR];
#pragma unroll
    for (int k = 0; k < CR; ++k) {
        const int64_t r = r0 + (int64_t)k * CNT;
        wv[k] = r < N ? W[r] : (T)0;
    }
    auto load = [&](T (&x)[CR], int l) {
        const T* Vl = Vc + (int64_t)l * N;
#pragma unroll
        for (int k = 0; k < CR; ++k) {
            const int64_t r = r0 + (int64_t)k * CNT;
            x[k] = r < N ? Vl[r] : (T)0;
        }
    };
    auto apply = [&](const T (&x)[CR], int l) {
        if constexpr (std::is_same<T, float>::value) {
            const float ch = cfh[l], cl = cfl[l];
#pragma unroll
            for (int k = 0; k < CR; ++k) wv[k] = fmaf(ch, x[k], fmaf(cl, x[k], wv[k]));
        } else {
            const double c = cf[l];
#pragma unroll
            for (int k = 0; k < CR; ++k) wv[k] = fma(-c, x[k], wv[k]);
        }
    };
    // the loads of vector l+1 are in flight while vector l is applied (rows
    // past N load 0 and are never stored)
    load(xa, 0);
    for (int l = 0; l <= j; l += 2) {
        if (l + 1 <= j) load(xb, l + 1);
        apply(xa, l);
        if (l + 1 > j) break;
        if (l + 2 <= j) load(xa, l + 2);
        apply(xb, l + 1);
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
static int64_t row_blocks(int64_t N) { return (N + CCHUNK_MIN - 1) / CCHUNK_MIN; }
template <typename T>
static int64_t row_blocks_t(int64_t N) {
    return (N + CNT * RowsPer<T>::v - 1) / (CNT * RowsPer<T>::v);
}
static int64_t spmv_blocks(int64_t N) {
    int64_t b = (N + CNT - 1) / CNT;
    return b > 152 * 16 ? 152 * 16 : b;
}

int64_t csr_scratch_slots(int64_t N, int m) {  // reduction partials per column
    const int64_t nb = row_blocks(N) > spmv_blocks(N) ? row_blocks(N) : spmv_blocks(N);
    return nb * 2 * (m + 1);
}

size_t csr_arnoldi_dev_bytes() { return sizeof(ArnoldiDev); }

// ------------------------------------------------------- SpMM dispatch --
template <typename T, int G, int LPR>
static void spmm_launch(const Prob* p, VecArgs<T> va, int xslot, int wslot, const int* aug, const ColState* st,
                        int j, int ncols, cudaStream_t s) {
    const Sys* sy = p->sys;
    const int64_t rows_per_block = CNT / LPR;
    int64_t gx = (p->N + rows_per_block - 1) / rows_per_block;
    if (gx > 152 * 16) gx = 152 * 16;
    dim3 grd((unsigned)gx, (unsigned)((ncols + G - 1) / G));
    k_spmm<T, G, LPR><<<grd, CNT, 0, s>>>(sy->d_rp, sy->d_col, (const T*)sy->d_val, sy->d_b, va, xslot, wslot,
                                          sy->n, p->N, aug, st, j, ncols);
}

template <typename T>
static bool spmm_dispatch(const Prob* p, int G, int LPR, VecArgs<T> va, int xslot, int wslot, const int* aug,
                          const ColState* st, int j, int ncols, cudaStream_t s) {
#define KV_SPMM_CASE(g, l)                                                  \
    if (G == g && LPR == l) {                                               \
        spmm_launch<T, g, l>(p, va, xslot, wslot, aug, st, j, ncols, s);    \
        return true;                                                        \
    }
    KV_SPMM_CASE(1, 1) KV_SPMM_CASE(1, 2) KV_SPMM_CASE(1, 4)
    KV_SPMM_CASE(2, 1) KV_SPMM_CASE(2, 2) KV_SPMM_CASE(2, 4)
    KV_SPMM_CASE(4, 1) KV_SPMM_CASE(4, 2) KV_SPMM_CASE(4, 4)
    KV_SPMM_CASE(8, 1) KV_SPMM_CASE(8, 2) KV_SPMM_CASE(8, 4)
#undef KV_SPMM_CASE
    return false;
}

// ----------------------------------------------------------- autotuner --
// Picks the SpMM group size G (columns per matrix read) and lanes per row
// for a CSR problem by timing every candidate on the problem's own buffers
// (CUDA events on the context stream) at problem creation.  Candidates keep
// the G input vectors of a group within about 96 MB so the column gathers
// stay in L2.  Results are cached in a text file (KV_AUTOTUNE_CACHE, default
// $HOME/.cache/kv_autotune.txt) keyed by device, rows, nonzeros, element size
// and column count.
static std::string tune_cache_path() {
    const char* e = getenv("KV_AUTOTUNE_CACHE");
    if (e && *e) return e;
    const char* h = getenv("HOME");
    return std::string(h ? h : "/tmp") + "/.cache/kv_autotune.txt";
}

static std::string tune_key(const Prob* p, int ncols) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, p->ctx->device);
    char buf[512];
    snprintf(buf, sizeof(buf), "%s|%d.%d|n=%lld|N=%lld|nnz=%lld|es=%zu|cols=%d", prop.name, prop.major, prop.minor,
             (long long)p->sys->n, (long long)p->N, (long long)p->sys->nnz, elem_size(p->prec), ncols);
    for (char* c = buf; *c; ++c)
        if (*c == ' ') *c = '_';
    return buf;
}

template <typename T>
static int autotune_t(Prob* p, int ncols, void* V) {
    const std::string key = tune_key(p, ncols);
    const std::string path = tune_cache_path();
    if (FILE* f = fopen(path.c_str(), "r")) {
        char k[512];
        int g, l;
        double us;
        while (fscanf(f, "%511s %d %d %lf", k, &g, &l, &us) == 4) {
            if (key == k) {
                p->spmm_G = g;
                p->spmm_LPR = l;
            }
        }
        fclose(f);
        if (p->spmm_G > 0) return KV_OK;
    }
    cudaStream_t s = p->ctx->stream;
    VecArgs<T> va{(T*)V, (int64_t)p->nvec * p->N};
    cudaEvent_t e0, e1;
    KV_CHECK_CUDA(cudaEventCreate(&e0));
    KV_CHECK_CUDA(cudaEventCreate(&e1));
    const double l2_budget = 96.0 * 1024 * 1024;
    double best = 1e30;
    int bg = 1, bl = 1;
    const int Gs[4] = {1, 2, 4, 8}, Ls[3] = {1, 2, 4};
    for (int gi = 0; gi < 4; ++gi) {
        const int G = Gs[gi];
        if (G > 1 && (G > ncols || (double)G * p->N * sizeof(T) > l2_budget)) continue;
        for (int li = 0; li < 3; ++li) {
            const int L = Ls[li];
            spmm_dispatch<T>(p, G, L, va, 0, 1, p->d_aug, p->d_state, 0, ncols, s);
            KV_CHECK_CUDA(cudaEventRecord(e0, s));
            for (int q = 0; q < 3; ++q) spmm_dispatch<T>(p, G, L, va, 0, 1, p->d_aug, p->d_state, 0, ncols, s);
            KV_CHECK_CUDA(cudaEventRecord(e1, s));
            KV_CHECK_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            KV_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                bg = G;
                bl = L;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    KV_CHECK_CUDA(cudaGetLastError());
    p->spmm_G = bg;
    p->spmm_LPR = bl;
    const std::string dir = path.substr(0, path.find_last_of('/'));
    (void)!system(("mkdir -p '" + dir + "' 2>/dev/null").c_str());
    if (FILE* f = fopen(path.c_str(), "a")) {
        fprintf(f, "%s %d %d %.3f\n", key.c_str(), bg, bl, best * 1000.0 / 3.0);
        fclose(f);
    }
    return KV_OK;
}

// Called by kv_problem for CSR problems whose Arnoldi columns run as one group.
int csr_autotune(Prob* p) {
    int narn = 0;
    for (int j = 0; j < p->i; ++j) narn += p->method[j] == KV_ARNOLDI;
    p->spmm_G = 0;
    p->spmm_LPR = 0;
    if (narn == 0) return KV_OK;
    if ((p->flags & KV_FLAG_NO_AUTOTUNE) || p->N < 65536) {  // small systems: a fixed choice
        p->spmm_G = narn >= 4 ? 4 : (narn >= 2 ? 2 : 1);
        p->spmm_LPR = 2;
        return KV_OK;
    }
    // the first Arnoldi column's vector set starts the timed group
    int j0 = 0;
    while (p->method[j0] != KV_ARNOLDI) ++j0;
    int run = 0;
    while (j0 + run < p->i && p->method[j0 + run] == KV_ARNOLDI) ++run;
    KV_CHECK_CUDA(cudaMemsetAsync(p->d_state, 0, sizeof(ColState) * (size_t)p->i, p->ctx->stream));
    void* V = (char*)p->d_vec + (size_t)j0 * p->nvec * p->N * elem_size(p->prec);
    const int rc = p->prec == KV_FP32 ? autotune_t<float>(p, run, V) : autotune_t<double>(p, run, V);
    return rc;
}

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
    dim3 gs((unsigned)spmv_blocks(N), (unsigned)ncols), gr((unsigned)row_blocks_t<T>(N), (unsigned)ncols);
    for (int it = 0; it < m; ++it) {
        if (lanczos) {
            const int vs = it % 3, ws = (it + 1) % 3, ps = (it + 2) % 3;
            {
                LaunchScope ls(p->ctx, "csr_spmv");
                k_spmv<T, true><<<gs, CNT, 0, st>>>(s->d_rp, s->d_col, (const T*)s->d_val, s->d_b, va, vs, ws, n, N,
                                                   aug, stp, H, m, it, partials, counters, nbx);
                KV_CHECK_CUDA(cudaGetLastError());
            }
            {
                LaunchScope ls(p->ctx, "csr_lanczos_update");
                if (it == 0)
                    k_lanczos3_update<T, true><<<gs, CNT, 0, st>>>(va, ws, vs, ps, N, stp, H, P, cd, m, it, partials,
                                                                  counters, nbx);
                else
                    k_lanczos3_update<T, false><<<gs, CNT, 0, st>>>(va, ws, vs, ps, N, stp, H, P, cd, m, it, partials,
                                                                   counters, nbx);
                KV_CHECK_CUDA(cudaGetLastError());
            }
            const int rc = launch_project(p, j0, ncols, (T*)V + (int64_t)ws * N, va.cstride, it + 1);
            if (rc) return rc;
        } else {
            if (p->spmm_G > 0 && !(p->flags & KV_FLAG_NO_SPMM)) {
                // grouped SpMM: the matrix is read once per group of spmm_G columns
                LaunchScope ls(p->ctx, "csr_spmm");
                if (!spmm_dispatch<T>(p, p->spmm_G, p->spmm_LPR, va, it, it + 1, aug, stp, it, ncols, st)) {
                    set_error("no SpMM kernel for G=%d LPR=%d", p->spmm_G, p->spmm_LPR);
                    return KV_EINVAL;
                }
                KV_CHECK_CUDA(cudaGetLastError());
            } else {
                LaunchScope ls(p->ctx, "csr_spmv");
                k_spmv<T, false><<<gs, CNT, 0, st>>>(s->d_rp, s->d_col, (const T*)s->d_val, s->d_b, va, it, it + 1, n,
                                                    N, aug, stp, H, m, it, partials, counters, nbx);
                KV_CHECK_CUDA(cudaGetLastError());
            }
            if (p->d_brow) {  // A'^T of the transpose dynamics: its last row b . x
                const int rc = launch_row_dot(p, j0, ncols, V, it, it + 1, it);
                if (rc) return rc;
            }
            {
                LaunchScope ls(p->ctx, "arnoldi_dots");
                k_arnoldi_dots<T><<<gr, CNT, 0, st>>>(va, N, stp, H, ad, m, it, partials, counters, nbx);
                KV_CHECK_CUDA(cudaGetLastError());
            }
            {
                LaunchScope ls(p->ctx, "arnoldi_update");
                const dim3 gu((unsigned)row_blocks(N), (unsigned)ncols);  // 8 rows per thread
                k_arnoldi_update<T><<<gu, CNT, 0, st>>>(va, N, stp, H, P, ad, cd, m, it, partials, counters, nbx);
                KV_CHECK_CUDA(cudaGetLastError());
            }
            const int rc = launch_project(p, j0, ncols, (T*)V + (int64_t)(it + 1) * N, va.cstride, it + 1);
            if (rc) return rc;
        }
        if (is_checkpoint(p, it + 1)) {
            const int rc = launch_error_check(p, j0, ncols, it + 1);
            if (rc) return rc;
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
