// k_csr.cu -- Krylov passes for sparse systems in CSR form.
//
// SpMV.  w = A' (s_j V_j) with A' = [[A, b], [0, 0]] when the state carries the
// constant-1 variable (Sec. 2.1): row r < n gets sum_e val[e] x[col[e]] +
// b[r] x[n], row n is zero.  One lane per row, the warp's entries staged in
// shared memory; the row sum is a double in the FP64 form and an error-free
// float pair (Dot2) in the FP32 form.
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
// The FP64 form forms the dots pass's products from exact float splits on
// the FP32 pipe (that pass is otherwise bound by the FP64 pipe); the update
// and the Lanczos passes keep FP64 arithmetic (moving their few FP64
// instructions off the pipe made them slower: latency, not the pipe, sets
// their time).
//
// Lanczos (Alg. 3) for symmetric CSR: SpMV fused with alpha_j = v_j . A v_j,
// then w = A v_j - alpha_j v_j - beta_j v_{j-1} over three rotating buffers.
//
// All scalars stay on the device; the last block of each pass finishes the
// deterministic reduction and writes them.
#include <errno.h>
#include <stdio.h>
#include <stdlib.h>
#include <sys/stat.h>

#include <string>
#include <type_traits>

#include "kv_internal.h"
#include "reduce.cuh"
#include "splits.cuh"

namespace kv {

constexpr int CNT = 256;           // threads per block
// rows per thread in the dots pass: 16 for the FP32 form (each basis
// vector's per-thread partials reduced across the warp as float pairs, so no
// FP64 instruction per vector), 8 for the FP64 form (its float splits of w and
// v_j take the registers of a second row set; 8 rows keep two blocks per SM)
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
constexpr int SPMV_STAGE = 256;  // matrix entries per warp staged in shared memory
template <typename T, bool ALPHA>
__global__ void __launch_bounds__(CNT, 6) k_spmv(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                              const T* __restrict__ val, const double* __restrict__ b,
                                              VecArgs<T> V, int xslot, int wslot, int64_t n, int64_t N,
                                              const int* aug, ColState* st, double* H, int m, int j,
                                              double* partials, unsigned* counters, int64_t nbx) {
    dep_wait();  // every input comes from the kernel before
    dep_release();
    const int cidx = blockIdx.y;
    ColState* s = st + cidx;
    if (s->done) return;
    const T* X = V.base + cidx * V.cstride + (int64_t)xslot * N;
    T* Wv = V.base + cidx * V.cstride + (int64_t)wslot * N;
    const double sj = s->s[j];
    const bool ag = aug[cidx] != 0;
    // one lane per row; the entries of the warp's 32 rows are contiguous in
    // the CSR arrays, so the warp stages them in shared memory with coalesced
    // loads (SPMV_STAGE at a time) and each lane walks its own row there, in
    // the order of the arrays
    __shared__ T sv[CNT / 32][SPMV_STAGE];
    __shared__ int32_t scol[CNT / 32][SPMV_STAGE];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double acc_alpha = 0.0;
    // warp-uniform loop over the warp's first row: every lane reaches every
    // shuffle and warp barrier
    for (int64_t rb = (int64_t)blockIdx.x * CNT + (threadIdx.x & ~31); rb < N; rb += (int64_t)gridDim.x * CNT) {
        const int64_t r = rb + lane;
        const bool inrow = r < n;
        // rows past n have the empty range at rp[n]
        const int64_t e0 = rp[inrow ? r : n], e1 = inrow ? rp[r + 1] : e0;
        const int64_t E0 = __shfl_sync(0xffffffffu, e0, 0), E1 = __shfl_sync(0xffffffffu, e1, 31);
        typename AccOf<T>::type d;
        for (int64_t base = E0; base < E1; base += SPMV_STAGE) {
            const int cnt = (int)(E1 - base < SPMV_STAGE ? E1 - base : SPMV_STAGE);
            for (int q = lane; q < cnt; q += 32) {
                sv[w][q] = val[base + q];
                scol[w][q] = col[base + q];
            }
            __syncwarp();
            const int lo = (int)((e0 > base ? e0 : base) - base);
            const int hi = (int)((e1 < base + cnt ? e1 : base + cnt) - base);
            // unrolled so that several gathers of the row are in flight at once
#pragma unroll 4
            for (int q = lo; q < hi; ++q) {
#ifdef KV_DEBUG
                // debug build: a matrix column outside [0, n) is skipped, not read
                if (scol[w][q] < 0 || scol[w][q] >= n) {
                    atomicOr(&s->status, KV_ST_INDEX);
                    continue;
                }
#endif
                d.add_prod(sv[w][q], X[scol[w][q]]);
            }
            __syncwarp();
        }
        if (r >= N) continue;
        double y = 0.0;  // the constant variable's row of A' is zero
        if (inrow) {
            y = d.value();
            if (ag && b) y = fma(b[r], (double)X[n], y);
            y *= sj;
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
//
// IL (interleaved input): the group's inputs come from xi, which holds row r
// of the group's G vectors side by side (xi[r * G + k] = X_k[r], G * size
// of T a multiple of 16 bytes), so the gather of row c for all G columns is
// one contiguous G-wide load (one 32-byte sector for 32 bytes) instead of G
// scattered ones.  k_interleave builds xi for every group from the
// column-major vectors just before the SpMM.
// One 32-byte read-only load (ld.global.nc.v8.b32, sm_100 and later): a
// lane's gather of a 32-byte row is one request instead of two 16-byte ones,
// and a warp's divergent gather costs the L1 about as much per request
// whatever its width up to 32 bytes.  The address is 32-byte aligned.
__device__ __forceinline__ void ld_nc_256(const void* p, uint32_t (&u)[8]) {
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
                 : "l"(p));
}

template <typename T, int G>
__device__ __forceinline__ void load_row(const T* __restrict__ src, T (&x)[G]) {
    static_assert((G * sizeof(T)) % 16 == 0, "interleaved rows are whole 16-byte words");
    constexpr int BYTES = (int)(G * sizeof(T));
    if constexpr (BYTES % 32 == 0) {  // rows of 32 or 64 bytes: 32-byte loads
        constexpr int W = BYTES / 32;
        uint32_t u[W][8];
#pragma unroll
        for (int q = 0; q < W; ++q) ld_nc_256(reinterpret_cast<const char*>(src) + 32 * q, u[q]);
#pragma unroll
        for (int q = 0; q < W; ++q) memcpy(&x[q * (32 / sizeof(T))], u[q], 32);
    } else {  // 16-byte rows
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(src));
        memcpy(&x[0], &w, 16);
    }
}

// error-free (float pairs) or plain (double) sum of the partial dot products
// of the LPR lanes that share a row, into the first of them
template <int LPR>
__device__ __forceinline__ void combine_lanes(Dot2f& d) {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, d.s, o, LPR);
        const float c2 = __shfl_down_sync(0xffffffffu, d.c, o, LPR);
        float t, err;
        two_sum_f(d.s, s2, t, err);
        d.s = t;
        d.c = __fadd_rn(__fadd_rn(d.c, c2), err);
    }
}
template <int LPR>
__device__ __forceinline__ void combine_lanes(Dot2d& d) {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) d.s += __shfl_down_sync(0xffffffffu, d.s, o, LPR);
}

constexpr int STAGE = 384;  // matrix entries per warp staged in shared memory (LPR = 0)

// LPR = 0 (staged): one lane per row; the warp's 32 rows have their entries
// contiguous in the CSR arrays, so the warp copies them to shared memory with
// coalesced loads (STAGE at a time) and each lane walks its own row there.
// With LPR >= 1 the lanes read their rows' entries directly.
template <typename T, int G, int LPR, bool IL>
__global__ void __launch_bounds__(CNT) k_spmm(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                              const T* __restrict__ val, const double* __restrict__ b, VecArgs<T> V,
                                              const T* __restrict__ xi, int xslot, int wslot, int64_t n, int64_t N,
                                              const int* aug, const ColState* st, int j, int ncols) {
    static_assert(G <= 32, "column flags are bit masks");
    using Acc = typename std::conditional<std::is_same<T, float>::value, Dot2f, Dot2d>::type;
    constexpr bool STAGED = LPR == 0;
    constexpr int LP = STAGED ? 1 : LPR;  // lanes per row
    const int cg0 = blockIdx.y * G;
    // the group's columns: X_k = xbase + k * cstride (or xg[. * G + k]), W_k = wbase + k * cstride
    const T* xbase = V.base + (int64_t)cg0 * V.cstride + (int64_t)xslot * N;
    const T* xg = IL ? xi + (int64_t)blockIdx.y * N * G : nullptr;
    T* wbase = V.base + (int64_t)cg0 * V.cstride + (int64_t)wslot * N;
    // live columns (inside the run, not broken down) and those that carry the
    // constant; the scales s_j and x[n] are read again in the epilogue, so the
    // loop keeps only accumulators and gathered values in registers
    unsigned act = 0, ag = 0;
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const int c = cg0 + k;
        if (c < ncols && !st[c].done) {
            act |= 1u << k;
            if (aug[c] != 0 && b) ag |= 1u << k;
        }
    }
    // x_k[c] for the G columns: one G-wide load (interleaved) or G loads
    // (column-major; dead slots read the group's first column)
    auto gather = [&](int c, T(&x)[G]) {
#ifdef KV_DEBUG
        // debug build: a matrix column outside [0, n) is skipped, not read
        if (c < 0 || c >= n) {
            atomicOr(&const_cast<ColState*>(st)[cg0].status, KV_ST_INDEX);
#pragma unroll
            for (int k = 0; k < G; ++k) x[k] = (T)0;
            return;
        }
#endif
        if constexpr (IL) {
            load_row<T, G>(xg + (int64_t)c * G, x);
        } else {
#pragma unroll
            for (int k = 0; k < G; ++k) x[k] = xbase[(((act >> k) & 1u) ? (int64_t)k * V.cstride : 0) + c];
        }
    };
    auto epilogue = [&](int k, int64_t r, bool inrow, double dot) {
        double y = 0.0;  // row n of A' (constant variable) is zero
        if (inrow) {
            y = dot;
            if ((ag >> k) & 1u) y = fma(b[r], (double)(IL ? xg[n * G + k] : xbase[(int64_t)k * V.cstride + n]), y);
        }
        wbase[k * V.cstride + r] = (T)(st[cg0 + k].s[j] * y);
    };
    const int lane = threadIdx.x & 31, sub = lane % LP;
    constexpr int WR = 32 / LP;  // rows per warp per step
    const int64_t gw = ((int64_t)blockIdx.x * CNT + threadIdx.x) >> 5;
    const int64_t nw = (int64_t)gridDim.x * (CNT / 32);
    // warp-uniform loop: every lane reaches every shuffle and warp barrier
    for (int64_t rb = gw * WR; rb < N; rb += nw * WR) {
        const int64_t r = rb + lane / LP;
        const bool inrow = r < n;
        Acc d[G];
        if constexpr (STAGED) {
            __shared__ T sv[CNT / 32][STAGE];
            __shared__ int32_t scol[CNT / 32][STAGE];
            const int w = threadIdx.x >> 5;
            // rows past n have the empty range at rp[n]
            const int64_t e0 = rp[inrow ? r : n], e1 = inrow ? rp[r + 1] : e0;
            const int64_t E0 = __shfl_sync(0xffffffffu, e0, 0), E1 = __shfl_sync(0xffffffffu, e1, 31);
            for (int64_t base = E0; base < E1; base += STAGE) {
                const int cnt = (int)(E1 - base < STAGE ? E1 - base : STAGE);
                for (int q = lane; q < cnt; q += 32) {
                    sv[w][q] = val[base + q];
                    scol[w][q] = col[base + q];
                }
                __syncwarp();
                const int lo = (int)((e0 > base ? e0 : base) - base);
                const int hi = (int)((e1 < base + cnt ? e1 : base + cnt) - base);
#pragma unroll 8
                for (int q = lo; q < hi; ++q) {
                    T x[G];
                    gather(scol[w][q], x);
                    const T v = sv[w][q];
#pragma unroll
                    for (int k = 0; k < G; ++k) d[k].add_prod(v, x[k]);
                }
                __syncwarp();
            }
        } else {
            const int64_t e0 = inrow ? rp[r] : 0, e1 = inrow ? rp[r + 1] : 0;
#pragma unroll 8
            for (int64_t e = e0 + sub; e < e1; e += LP) {
                T x[G];
                gather(col[e], x);
                const T v = val[e];
#pragma unroll
                for (int k = 0; k < G; ++k) d[k].add_prod(v, x[k]);
            }
#pragma unroll
            for (int k = 0; k < G; ++k) combine_lanes<LP>(d[k]);
        }
        if (sub == 0 && r < N) {
#pragma unroll
            for (int k = 0; k < G; ++k)
                if ((act >> k) & 1u) epilogue(k, r, inrow, d[k].value());
        }
    }
}

// xi[g][r][k] = X_{g G + k}[r] (slot xslot of column g G + k; zero past the
// run): one thread per row, G column reads coalesced across the warp, one
// contiguous G-wide store.  blockIdx.y = group.
template <typename T, int G>
__global__ void __launch_bounds__(CNT) k_interleave(VecArgs<T> V, int xslot, int64_t N, int ncols, T* __restrict__ xi) {
    static_assert((G * sizeof(T)) % 16 == 0, "interleaved rows are whole 16-byte words");
    const int cg0 = blockIdx.y * G;
    const T* x0 = V.base + (int64_t)cg0 * V.cstride + (int64_t)xslot * N;
    T* out = xi + (int64_t)blockIdx.y * N * G;
    const int nk = ncols - cg0 < G ? ncols - cg0 : G;
    for (int64_t r = (int64_t)blockIdx.x * CNT + threadIdx.x; r < N; r += (int64_t)gridDim.x * CNT) {
        T v[G];
#pragma unroll
        for (int k = 0; k < G; ++k) v[k] = k < nk ? x0[k * V.cstride + r] : T(0);
        uint4* o4 = reinterpret_cast<uint4*>(out + r * G);
#pragma unroll
        for (int q = 0; q < (int)(G * sizeof(T) / 16); ++q) {
            uint4 w;
            memcpy(&w, v + q * (16 / sizeof(T)), 16);
            o4[q] = w;
        }
    }
}

// gather of C x by a whole block; result in thread 0
template <typename T>
__device__ double cgather(const CDesc& cd, int r, const T* x, double* sh, int* status) {
    double v = 0.0;
    for (int64_t e = cd.rp[r] + threadIdx.x; e < cd.rp[r + 1]; e += CNT) v += c_entry(cd, e, x, status);
    return block_sum<CNT>(v, sh);
}

// Shared epilogue of every pass that produces w = unnormalised v_{j+1}:
// beta = ||w||, breakdown test against ||A v_j||^2 = sum_l H[l][j]^2 + beta^2,
// scale, H entries, P column.  Runs in the last block, all threads.  hcol2 >= 0
// is sum_l H[l][j]^2 already known to the caller (else read from H); cw, when
// given, holds C w for the o rows of C (already reduced over the grid), else
// the block gathers it.
template <typename T>
__device__ void finish_vector(double nw2, const T* W, ColState* s, double* H, double* P, const CDesc& cd, int m,
                              int j, bool symmetric, double* sh, double hcol2 = -1.0, const double* cw = nullptr) {
    __shared__ double snext;
    __shared__ int cont;
    if (threadIdx.x == 0) {
        const double beta = sqrt(nw2);
        H[(int64_t)(j + 1) * m + j] = beta;
        double nav2 = beta * beta;
        if (hcol2 >= 0.0) {
            nav2 += hcol2;
        } else {
            // Lanczos: column j of H has entries in rows j-1 and j only (the
            // rest stay zero), so one thread need not walk the whole column
            for (int l = symmetric && j > 0 ? j - 1 : 0; l <= j; ++l)
                nav2 += H[(int64_t)l * m + j] * H[(int64_t)l * m + j];
        }
        if (!(beta > 1e-12 * sqrt(nav2)) || !isfinite(beta)) {
            if (!isfinite(beta)) s->status |= KV_ST_NONFINITE;
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
    if (cw) {
        if (threadIdx.x < cd.o) P[(int64_t)threadIdx.x * m + (j + 1)] = snext * cw[threadIdx.x];
        return;
    }
    for (int r = 0; r < cd.o; ++r) {
        const double v = cgather<T>(cd, r, W, sh, &s->status);
        if (threadIdx.x == 0) P[(int64_t)r * m + (j + 1)] = snext * v;
    }
}

// C w of the Lanczos update folded into its grid reduction: with at most
// CINL_ROWS rows and CNT entries in C, each block adds up the entries whose
// column it wrote itself, and the last block only sums the blocks' shares
// (no gather after the grid reduction).
constexpr int CINL_ROWS = 4;

// ------------------------------------------------------ Lanczos update --
template <typename T, bool FIRST>
__global__ void __launch_bounds__(CNT, 4) k_lanczos3_update(VecArgs<T> V, int wslot, int vslot, int pslot, int64_t N,
                                                         ColState* st, double* Hall, double* Pall, CDesc cd, int cinl,
                                                         int m, int j, double* partials, unsigned* counters,
                                                         int64_t nbx) {
    dep_wait();  // every input comes from the kernel before
    dep_release();
    const int cidx = blockIdx.y;
    ColState* s = st + cidx;
    if (s->done) return;
    double* H = Hall + (int64_t)cidx * (m + 1) * m;
    T* Wv = V.base + cidx * V.cstride + (int64_t)wslot * N;
    const T* Vj = V.base + cidx * V.cstride + (int64_t)vslot * N;
    const T* Vp = V.base + cidx * V.cstride + (int64_t)pslot * N;
    const double alpha = H[(int64_t)j * m + j];
    const double ca = -alpha * s->s[j];
    const double hb = FIRST ? 0.0 : H[(int64_t)j * m + (j - 1)];  // beta_j = H[j-1][j]
    const double cb = -hb * (FIRST ? 0.0 : s->s[j - 1]);
    typename AccOf<T>::type acc;
    // four rows per thread per round, all their loads issued before the
    // arithmetic (the three vectors are distinct buffers)
    const int64_t stride = (int64_t)gridDim.x * CNT;
    int64_t r = (int64_t)blockIdx.x * CNT + threadIdx.x;
    for (; r + 3 * stride < N; r += 4 * stride) {
        T wv[4], vj[4], vp[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            wv[k] = Wv[r + k * stride];
            vj[k] = __ldcs(Vj + r + k * stride);
            vp[k] = FIRST ? (T)0 : __ldcs(Vp + r + k * stride);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double w = fma(ca, (double)vj[k], (double)wv[k]);
            if (!FIRST) w = fma(cb, (double)vp[k], w);
            const T wt = (T)w;
            Wv[r + k * stride] = wt;
            acc.add_prod(wt, wt);
        }
    }
    for (; r < N; r += stride) {
        double w = fma(ca, (double)Vj[r], (double)Wv[r]);
        if (!FIRST) w = fma(cb, (double)Vp[r], w);
        const T wt = (T)w;
        Wv[r] = wt;
        acc.add_prod(wt, wt);
    }
    __shared__ double sh[CNT / 32];
    __shared__ int flag;
    __shared__ double cw[CINL_ROWS];
    const double part = block_sum<CNT>(acc.value(), sh);  // its barriers also publish the block's W
    // column region: ||w||^2 partials, then (cinl) one row of partials per row of C
    double* preg = partials + (int64_t)cidx * nbx * (cinl ? 1 + CINL_ROWS : 1);
    if (cinl) {
        // row c of W was written by block (c mod stride) / CNT
        const int64_t e0 = cd.rp[0], ne = cd.rp[cd.o] - e0;
        double v = 0.0;
        int row = -1;
        if (threadIdx.x < ne) {
            const int64_t e = e0 + threadIdx.x, c = cd.col[e];
            if (c < 0 || c >= cd.n) {
                if (blockIdx.x == 0) atomicOr(&s->status, KV_ST_INDEX);  // skipped, not read
            } else if ((c % stride) / CNT == blockIdx.x) {
                row = 0;
                while (cd.rp[row + 1] <= e) ++row;
                v = cd.val[e] * (double)__ldcg(Wv + c);
            }
        }
        if (__syncthreads_or(row >= 0)) {
            for (int q = 0; q < cd.o; ++q) {
                const double r = block_sum<CNT>(row == q ? v : 0.0, sh);
                if (threadIdx.x == 0) preg[(int64_t)(1 + q) * nbx + blockIdx.x] = r;
            }
        } else if (threadIdx.x == 0) {
            for (int q = 0; q < cd.o; ++q) preg[(int64_t)(1 + q) * nbx + blockIdx.x] = 0.0;
        }
        // thread 0 wrote every partial of the block: grid_arrive's fence covers them
    }
    if (!grid_arrive(part, preg, counters + cidx, blockIdx.x, gridDim.x, &flag)) return;
    const double tot = grid_finish<CNT>(preg, gridDim.x, counters + cidx, sh);
    if (cinl) {
        for (int q = 0; q < cd.o; ++q) {
            double v = 0.0;
            for (int64_t b = threadIdx.x; b < gridDim.x; b += CNT) v += __ldcg(preg + (int64_t)(1 + q) * nbx + b);
            v = block_sum<CNT>(v, sh);
            if (threadIdx.x == 0) cw[q] = v;
        }
        __syncthreads();
    }
    // the column of H above beta: alpha_j and beta_j, both already here
    finish_vector<T>(tot, Wv, s, H, Pall + (int64_t)cidx * cd.o * m, cd, m, j, true, sh, alpha * alpha + hb * hb,
                     cinl ? cw : nullptr);
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
    // FP64 form: the products are formed on the FP32 pipe from float splits
    // (splits.cuh; this pass is bound by the FP64 pipe otherwise), each value
    // x held as x1 + x2 (24 exact leading bits, the rest rounded to a float:
    // 2^-48 of x) at a power-of-two scale: basis vector l by 2^(1-E(s_l))
    // (|V_l| <= ||V_l|| = 1/s_l), v_j likewise, w by the warp's largest
    // exponent.  Per (basis vector, warp) the float-pair sums become doubles
    // once, rescaled.
    constexpr bool SPLIT = std::is_same<T, double>::value;
    auto exp_of = [](double x) { return (int)(((unsigned)__double2hiint(x) >> 20) & 0x7ffu); };
    auto sh_of_scale = [&](double sc) { return 1 - (exp_of(sc) - 1023); };  // 1/sc < 2^result
    float wh[SPLIT ? CR : 1], wl[SPLIT ? CR : 1], vh[SPLIT ? CR : 1], vl[SPLIT ? CR : 1];
    int shw = 0, shv = 0;
    if constexpr (SPLIT) {
        int ew = 0;
#pragma unroll
        for (int k = 0; k < CR; ++k) ew = max(ew, exp_of(wv[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ew = max(ew, __shfl_xor_sync(0xffffffffu, ew, o));
        shw = ew - 1023 + 1;  // |w| < 2^shw over the warp
        shv = sh_of_scale(s->s[j]);
#pragma unroll
        for (int k = 0; k < CR; ++k) {
            const F2 a = split2((double)wv[k], shw), b = split2((double)vv[k], shv);
            wh[k] = a.a1;
            wl[k] = a.a2;
            vh[k] = b.a1;
            vl[k] = b.a2;
        }
    }
    auto load = [&](T (&x)[CR], int l) {
        const T* Vl = Vc + (int64_t)l * N;
#pragma unroll
        for (int k = 0; k < CR; ++k) {
            const int64_t r = r0 + (int64_t)k * CNT;
            x[k] = r < N ? Vl[r] : (T)0;
        }
    };
    // this thread's products with basis vector l
    auto prod = [&](const T (&x)[CR], T& at, T& gt) {
        at = 0;
        gt = 0;
#pragma unroll
        for (int k = 0; k < CR; ++k) {
            at = fma(x[k], wv[k], at);
            gt = fma(x[k], vv[k], gt);
        }
    };
    // the four sums of basis vectors l and l+1 (h1 and g of each) over the
    // warp by a transposed butterfly: at the first two levels each lane
    // hands half of what it holds to its partner, so the five levels cost 6
    // additions instead of 20; lanes 0, 8, 16, 24 end with the four totals.
    // FP32 form: float pairs (hi, lo) combined error-free; FP64: doubles.
    auto reduce4 = [&](T a0, T g0, T a1, T g1, int l, bool two) {
        const bool up = lane & 16, mid = lane & 8;
        if constexpr (std::is_same<T, float>::value) {
            float kh0 = up ? a1 : a0, kh1 = up ? g1 : g0, kl0 = 0.f, kl1 = 0.f;
            const float s0 = up ? a0 : a1, s1 = up ? g0 : g1;
            {
                float t, e;
                two_sum_f(kh0, __shfl_xor_sync(0xffffffffu, s0, 16), t, e);
                kh0 = t;
                kl0 = e;
                two_sum_f(kh1, __shfl_xor_sync(0xffffffffu, s1, 16), t, e);
                kh1 = t;
                kl1 = e;
            }
            float h = mid ? kh1 : kh0, lo = mid ? kl1 : kl0;
            {
                const float sh = mid ? kh0 : kh1, sl = mid ? kl0 : kl1;
                const float rh = __shfl_xor_sync(0xffffffffu, sh, 8);
                const float rl = __shfl_xor_sync(0xffffffffu, sl, 8);
                float t, e;
                two_sum_f(h, rh, t, e);
                h = t;
                lo = __fadd_rn(__fadd_rn(lo, rl), e);
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                const float rh = __shfl_xor_sync(0xffffffffu, h, o);
                const float rl = __shfl_xor_sync(0xffffffffu, lo, o);
                float t, e;
                two_sum_f(h, rh, t, e);
                h = t;
                lo = __fadd_rn(__fadd_rn(lo, rl), e);
            }
            if ((lane & 7) == 0 && (two || !up)) {
                const int q = (up ? l + 1 : l) + (mid ? KV_MAX_M + 1 : 0);
                wsumf[q][warp] = make_float2(h, lo);
            }
        } else {
            double k0 = up ? a1 : a0, k1 = up ? g1 : g0;
            k0 += __shfl_xor_sync(0xffffffffu, up ? a0 : a1, 16);
            k1 += __shfl_xor_sync(0xffffffffu, up ? g0 : g1, 16);
            double x = (mid ? k1 : k0) + __shfl_xor_sync(0xffffffffu, mid ? k0 : k1, 8);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if ((lane & 7) == 0 && (two || !up)) {
                const int q = (up ? l + 1 : l) + (mid ? KV_MAX_M + 1 : 0);
                wsum[q][warp] = x;
            }
        }
    };
    // FP64 form: this thread's products with basis vector l as float pairs
    // (TwoProduct of the leading parts, the cross terms in the low word,
    // compensated additions)
    auto prod_split = [&](const T (&x)[CR], int shx, float& ah, float& al, float& gh, float& gl) {
        ah = al = gh = gl = 0.f;
#pragma unroll
        for (int k = 0; k < CR; ++k) {
            const F2 xs = split2((double)x[k], shx);
            const float x1 = xs.a1, x2 = xs.a2;
            float t, e;
            const float pa = __fmul_rn(x1, wh[k]);
            const float ea = __fmaf_rn(x1, wh[k], -pa);
            const float ca = __fmaf_rn(x1, wl[k], __fmul_rn(x2, wh[k]));
            two_sum(ah, pa, t, e);
            ah = t;
            al = __fadd_rn(al, __fadd_rn(e, __fadd_rn(ea, ca)));
            const float pg = __fmul_rn(x1, vh[k]);
            const float eg = __fmaf_rn(x1, vh[k], -pg);
            const float cg = __fmaf_rn(x1, vl[k], __fmul_rn(x2, vh[k]));
            two_sum(gh, pg, t, e);
            gh = t;
            gl = __fadd_rn(gl, __fadd_rn(e, __fadd_rn(eg, cg)));
        }
    };
    // the same transposed butterfly as reduce4 on float pairs; the four totals
    // become doubles at their scales in wsum
    auto reduce4p = [&](float ah0, float al0, float gh0, float gl0, float ah1, float al1, float gh1, float gl1,
                        int l, bool two, int shx0, int shx1) {
        const bool up = lane & 16, mid = lane & 8;
        float kh0 = up ? ah1 : ah0, kl0 = up ? al1 : al0, kh1 = up ? gh1 : gh0, kl1 = up ? gl1 : gl0;
        const float s0h = up ? ah0 : ah1, s0l = up ? al0 : al1, s1h = up ? gh0 : gh1, s1l = up ? gl0 : gl1;
        {
            float t, e;
            const float r0h = __shfl_xor_sync(0xffffffffu, s0h, 16), r0l = __shfl_xor_sync(0xffffffffu, s0l, 16);
            const float r1h = __shfl_xor_sync(0xffffffffu, s1h, 16), r1l = __shfl_xor_sync(0xffffffffu, s1l, 16);
            two_sum_f(kh0, r0h, t, e);
            kh0 = t;
            kl0 = __fadd_rn(__fadd_rn(kl0, r0l), e);
            two_sum_f(kh1, r1h, t, e);
            kh1 = t;
            kl1 = __fadd_rn(__fadd_rn(kl1, r1l), e);
        }
        float h = mid ? kh1 : kh0, lo = mid ? kl1 : kl0;
        {
            const float sh = mid ? kh0 : kh1, sl = mid ? kl0 : kl1;
            const float rh = __shfl_xor_sync(0xffffffffu, sh, 8);
            const float rl = __shfl_xor_sync(0xffffffffu, sl, 8);
            float t, e;
            two_sum_f(h, rh, t, e);
            h = t;
            lo = __fadd_rn(__fadd_rn(lo, rl), e);
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            const float rh = __shfl_xor_sync(0xffffffffu, h, o);
            const float rl = __shfl_xor_sync(0xffffffffu, lo, o);
            float t, e;
            two_sum_f(h, rh, t, e);
            h = t;
            lo = __fadd_rn(__fadd_rn(lo, rl), e);
        }
        if ((lane & 7) == 0 && (two || !up)) {
            const int q = (up ? l + 1 : l) + (mid ? KV_MAX_M + 1 : 0);
            wsum[q][warp] = ldexp((double)h + (double)lo, (up ? shx1 : shx0) + (mid ? shv : shw));
        }
    };
    // two register buffers: the loads of the next vectors are in flight while
    // the products of the current ones are formed and reduced
    load(xa, 0);
    for (int l = 0; l <= j; l += 2) {
        const bool two = l + 1 <= j;
        if (two) load(xb, l + 1);
        if constexpr (SPLIT) {
            const int shx0 = sh_of_scale(s->s[l]), shx1 = two ? sh_of_scale(s->s[l + 1]) : 0;
            float ah0, al0, gh0, gl0, ah1 = 0.f, al1 = 0.f, gh1 = 0.f, gl1 = 0.f;
            prod_split(xa, shx0, ah0, al0, gh0, gl0);
            if (l + 2 <= j) load(xa, l + 2);
            if (two) prod_split(xb, shx1, ah1, al1, gh1, gl1);
            reduce4p(ah0, al0, gh0, gl0, ah1, al1, gh1, gl1, l, two, shx0, shx1);
        } else {
            T a0, g0, a1 = 0, g1 = 0;
            prod(xa, a0, g0);
            if (l + 2 <= j) load(xa, l + 2);
            if (two) prod(xb, a1, g1);
            reduce4(a0, g0, a1, g1, l, two);
        }
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
    return b > 152 * 8 ? 152 * 8 : b;
}
// k_spmv: one wave at the 6 blocks per SM its launch bounds guarantee (40
// registers a thread); at most spmv_blocks
static int64_t spmv_grid(int64_t N) {
    int64_t b = (N + CNT - 1) / CNT;
    return b > 152 * 6 ? 152 * 6 : b;
}
// k_lanczos3_update: one wave at its 4 blocks per SM (four rows a thread in
// flight need the registers)
static int64_t update_grid(int64_t N) {
    int64_t b = (N + CNT - 1) / CNT;
    return b > 152 * 4 ? 152 * 4 : b;
}

int64_t csr_scratch_slots(int64_t N, int m) {  // reduction partials per column
    const int64_t nb = row_blocks(N) > spmv_blocks(N) ? row_blocks(N) : spmv_blocks(N);
    return nb * 2 * (m + 1);
}

size_t csr_arnoldi_dev_bytes() { return sizeof(ArnoldiDev); }

// ------------------------------------------------------- SpMM dispatch --
// Grid-stride kernels get one full wave: the SMs times the blocks of CNT
// threads that fit on one SM at the kernel's register count.  Each kernel's
// wave is found once, on the device of the first problem that sizes it (one
// GPU model per process).
template <typename K>
static int64_t one_wave(K kernel, int device) {
    int nb = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, CNT, 0) != cudaSuccess || nb < 1) nb = 1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || nsm < 1) nsm = 152;
    return (int64_t)nb * nsm;
}

// warm_only: size the grids (occupancy queries, once per kernel) and launch
// nothing; done when the problem is created, so that no query runs inside a
// stream capture.
template <typename T, int G, int LPR, bool IL>
static void spmm_launch(const Prob* p, VecArgs<T> va, int xslot, int wslot, const int* aug, const ColState* st,
                        int j, int ncols, cudaStream_t s, bool warm_only) {
    static const int64_t wave = one_wave(k_spmm<T, G, LPR, IL>, p->ctx->device);
    static const int64_t iwave = IL ? one_wave(k_interleave<T, IL ? G : 16 / sizeof(T)>, p->ctx->device) : 0;
    if (warm_only) return;
    const Sys* sy = p->sys;
    const int64_t rows_per_block = CNT / (LPR > 0 ? LPR : 1);
    int64_t gx = (p->N + rows_per_block - 1) / rows_per_block;
    if (gx > wave) gx = wave;
    const unsigned ng = (unsigned)((ncols + G - 1) / G);
    if constexpr (IL) {  // the groups' inputs, row-interleaved, first
        int64_t gi = (p->N + CNT - 1) / CNT;
        if (gi > iwave) gi = iwave;
        k_interleave<T, G><<<dim3((unsigned)gi, ng), CNT, 0, s>>>(va, xslot, p->N, ncols, (T*)p->d_xi);
    }
    k_spmm<T, G, LPR, IL><<<dim3((unsigned)gx, ng), CNT, 0, s>>>(sy->d_rp, sy->d_col, (const T*)sy->d_val, sy->d_b,
                                                                  va, (const T*)p->d_xi, xslot, wslot, sy->n, p->N,
                                                                  aug, st, j, ncols);
}

// Interleaved group widths: 16, 32 and 64 bytes per row.
template <typename T>
struct IlWidths {
    static constexpr int g[3] = {16 / (int)sizeof(T), 32 / (int)sizeof(T), 64 / (int)sizeof(T)};
};

// G > 0: column-major gathers; G < 0: groups of -G columns from the
// interleaved copy (built in the same call)
template <typename T>
static bool spmm_dispatch(const Prob* p, int G, int LPR, VecArgs<T> va, int xslot, int wslot, const int* aug,
                          const ColState* st, int j, int ncols, cudaStream_t s, bool warm_only = false) {
#define KV_SPMM_CASE(g, l, il)                                                          \
    if (G == (il ? -(g) : (g)) && LPR == l) {                                           \
        spmm_launch<T, g, l, il>(p, va, xslot, wslot, aug, st, j, ncols, s, warm_only); \
        return true;                                                                    \
    }
    KV_SPMM_CASE(1, 1, false) KV_SPMM_CASE(1, 2, false) KV_SPMM_CASE(1, 4, false)
    KV_SPMM_CASE(2, 1, false) KV_SPMM_CASE(2, 2, false) KV_SPMM_CASE(2, 4, false)
    KV_SPMM_CASE(4, 1, false) KV_SPMM_CASE(4, 2, false) KV_SPMM_CASE(4, 4, false)
    KV_SPMM_CASE(8, 1, false) KV_SPMM_CASE(8, 2, false) KV_SPMM_CASE(8, 4, false)
    constexpr int g0 = IlWidths<T>::g[0], g1 = IlWidths<T>::g[1], g2 = IlWidths<T>::g[2];
    if (p->d_xi) {
        KV_SPMM_CASE(g0, 0, true) KV_SPMM_CASE(g0, 1, true) KV_SPMM_CASE(g0, 2, true)
        KV_SPMM_CASE(g1, 0, true) KV_SPMM_CASE(g1, 1, true) KV_SPMM_CASE(g1, 2, true)
        KV_SPMM_CASE(g2, 0, true) KV_SPMM_CASE(g2, 1, true) KV_SPMM_CASE(g2, 2, true)
    }
#undef KV_SPMM_CASE
    return false;
}

// ----------------------------------------------------------- autotuner --
// Picks the SpMM form (column-major gathers, or gathers from the interleaved
// copy with the interleave pass counted), the group size G (columns per
// matrix read) and lanes per row for a CSR problem by timing every candidate
// on the problem's own buffers (CUDA events on the context stream) at problem
// creation.  Results are cached in a text file (KV_AUTOTUNE_CACHE, default
// $HOME/.cache/kv_autotune.txt; one line "key G LPR microseconds", G < 0 for
// the interleaved form) keyed by device, rows, nonzeros, element size and
// column count.
static std::string tune_cache_path() {
    const char* e = getenv("KV_AUTOTUNE_CACHE");
    if (e && *e) return e;
    const char* h = getenv("HOME");
    return std::string(h ? h : "/tmp") + "/.cache/kv_autotune.txt";
}

// mkdir -p of the cache file's directory, without a shell (the path comes
// from the environment); failures only mean the result is not cached.
static void make_dirs(const std::string& dir) {
    for (size_t k = 1; k <= dir.size(); ++k)
        if (k == dir.size() || dir[k] == '/') {
            const std::string d = dir.substr(0, k);
            if (mkdir(d.c_str(), 0755) != 0 && errno != EEXIST) return;
        }
}

static std::string tune_key(const Prob* p, int ncols) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, p->ctx->device);
    char buf[512];
    snprintf(buf, sizeof(buf), "%s|%d.%d|n=%lld|N=%lld|nnz=%lld|es=%zu|cols=%d|il", prop.name, prop.major, prop.minor,
             (long long)p->sys->n, (long long)p->N, (long long)p->sys->nnz, elem_size(p->prec), ncols);
    for (char* c = buf; *c; ++c)
        if (*c == ' ') *c = '_';
    return buf;
}

// The autotuner's candidates keep a group's inputs within about 96 MB so its
// gathers stay in L2.  Interleaved widths larger than the smallest one are
// tried only when the smallest would need more than one group.
constexpr double L2_BUDGET = 96.0 * 1024 * 1024;
static bool plain_candidate(int G, int64_t N, size_t es, int ncols) {
    return G == 1 || (G <= ncols && (double)G * N * es <= L2_BUDGET);
}
static bool il_candidate(int G, int g0, int64_t N, size_t es, int ncols) {
    return (double)G * N * es <= L2_BUDGET && (G == g0 || G / 2 < ncols);
}
static int il_width(size_t es, int q) { return (16 << q) / (int)es; }  // q = 0, 1, 2

static bool autotuned(const Prob* p) {
    return !(p->flags & (KV_FLAG_NO_AUTOTUNE | KV_FLAG_NO_SPMM)) && p->N >= 65536;
}

// KV_SPMM_SHAPE="G,LPR" fixes the SpMM shape of every CSR Arnoldi problem
// created afterwards (G < 0: interleaved groups of -G columns); for tests and
// measurements.  Returns false when unset or not a shape that exists.
static bool forced_shape(size_t es, int* G, int* L) {
    const char* e = getenv("KV_SPMM_SHAPE");
    if (!e || sscanf(e, "%d,%d", G, L) != 2) return false;
    if (*G > 0) return (*G == 1 || *G == 2 || *G == 4 || *G == 8) && (*L == 1 || *L == 2 || *L == 4);
    if (*L != 0 && *L != 1 && *L != 2) return false;
    for (int q = 0; q < 3; ++q)
        if (-*G == il_width(es, q)) return true;
    return false;
}

static int longest_arnoldi_run(const Prob* p) {  // one SpMM group set per run
    int run = 0;
    for (int j = 0, r = 0; j < p->i; ++j) {
        r = p->method[j] == KV_ARNOLDI ? r + 1 : 0;
        run = r > run ? r : run;
    }
    return run;
}

size_t csr_xi_bytes(const Prob* p) {
    if (p->sys->kind != 1 || (p->flags & KV_FLAG_NO_SPMM)) return 0;
    const int run = longest_arnoldi_run(p);
    if (run == 0) return 0;
    const size_t es = elem_size(p->prec);
    int fg, fl;
    if (forced_shape(es, &fg, &fl)) return fg < 0 ? (size_t)((run - fg - 1) / -fg) * -fg * p->N * es : 0;
    if (!autotuned(p)) return 0;
    size_t best = 0;
    for (int q = 0; q < 3; ++q) {
        const int G = il_width(es, q);
        if (!il_candidate(G, il_width(es, 0), p->N, es, run)) continue;
        const size_t b = (size_t)((run + G - 1) / G) * G * p->N * es;
        best = b > best ? b : best;
    }
    return best;
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
            if (key == k && (g > 0 || p->d_xi)) {
                p->spmm_G = g;
                p->spmm_LPR = l;
            }
        }
        fclose(f);
        if (p->spmm_G != 0) return KV_OK;
    }
    cudaStream_t s = p->ctx->stream;
    VecArgs<T> va{(T*)V, (int64_t)p->nvec * p->N};
    cudaEvent_t e0, e1;
    KV_CHECK_CUDA(cudaEventCreate(&e0));
    KV_CHECK_CUDA(cudaEventCreate(&e1));
    double best = 1e30;
    int bg = 1, bl = 1;
    const int Ls[4] = {0, 1, 2, 4};  // 0: staged rows (interleaved form only)
    std::vector<int> cand;  // signed group sizes: > 0 column-major, < 0 interleaved
    for (int G : {1, 2, 4, 8})
        if (plain_candidate(G, p->N, sizeof(T), ncols)) cand.push_back(G);
    if (p->d_xi)
        for (int q = 0; q < 3; ++q) {
            const int G = il_width(sizeof(T), q);
            if (il_candidate(G, il_width(sizeof(T), 0), p->N, sizeof(T), ncols)) cand.push_back(-G);
        }
    for (int G : cand) {
        for (int li = 0; li < 4; ++li) {
            const int L = Ls[li];
            if (!spmm_dispatch<T>(p, G, L, va, 0, 1, p->d_aug, p->d_state, 0, ncols, s)) continue;
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
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos && slash > 0) make_dirs(path.substr(0, slash));
    if (FILE* f = fopen(path.c_str(), "a")) {
        fprintf(f, "%s %d %d %.3f\n", key.c_str(), bg, bl, best * 1000.0 / 3.0);
        fclose(f);
    }
    return KV_OK;
}

static int choose_shape(Prob* p) {
    int narn = 0;
    for (int j = 0; j < p->i; ++j) narn += p->method[j] == KV_ARNOLDI;
    p->spmm_G = 0;
    p->spmm_LPR = 0;
    if (narn == 0) return KV_OK;
    int fg, fl;
    if (!(p->flags & KV_FLAG_NO_SPMM) && forced_shape(elem_size(p->prec), &fg, &fl)) {
        p->spmm_G = fg;
        p->spmm_LPR = fl;
        return KV_OK;
    }
    if (!autotuned(p)) {  // small systems, or asked for: a fixed choice
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
    return p->prec == KV_FP32 ? autotune_t<float>(p, run, V) : autotune_t<double>(p, run, V);
}

// Called by kv_problem for CSR problems: picks the SpMM shape of the Arnoldi
// columns and sizes its grids.
int csr_autotune(Prob* p) {
    const int rc = choose_shape(p);
    if (rc || p->spmm_G == 0) return rc;
    const bool ok = p->prec == KV_FP32
                        ? spmm_dispatch<float>(p, p->spmm_G, p->spmm_LPR, {}, 0, 0, nullptr, nullptr, 0, 0, 0, true)
                        : spmm_dispatch<double>(p, p->spmm_G, p->spmm_LPR, {}, 0, 0, nullptr, nullptr, 0, 0, 0, true);
    if (!ok) {
        set_error("no SpMM kernel for G=%d LPR=%d", p->spmm_G, p->spmm_LPR);
        return KV_EINVAL;
    }
    return KV_OK;
}

template <typename T>
static int run_csr_column_t(Prob* p, int j0, int ncols, void* V, ArnoldiDev* ad, bool lanczos) {
    const Sys* s = p->sys;
    const int64_t N = p->N, n = s->n;
    cudaStream_t st = p->ctx->stream;
    VecArgs<T> va{(T*)V, (int64_t)p->nvec * N};
    const int m = p->m;
    CDesc cd{p->o, p->d_crp, p->d_ccol, p->d_cval, p->N};
    ColState* stp = p->d_state + j0;
    double* H = p->d_H + (int64_t)j0 * (m + 1) * m;
    double* P = p->d_P + (int64_t)j0 * p->o * m;
    int* aug = p->d_aug + j0;
    const int64_t nbx = row_blocks(N) > spmv_blocks(N) ? row_blocks(N) : spmv_blocks(N);
    double* partials = p->red.partials;
    unsigned* counters = p->d_counters;
    dim3 gs((unsigned)spmv_blocks(N), (unsigned)ncols), gr((unsigned)row_blocks_t<T>(N), (unsigned)ncols);
    const dim3 gv((unsigned)spmv_grid(N), (unsigned)ncols), gu((unsigned)update_grid(N), (unsigned)ncols);
    // C w inside the update's reduction: few rows and entries, and room for
    // 1 + CINL_ROWS rows of partials in a column's 2 (m + 1) (csr_scratch_slots)
    const int cinl = p->o >= 1 && p->o <= CINL_ROWS && p->c_nnz <= CNT && 1 + CINL_ROWS <= 2 * (m + 1) ? 1 : 0;
    for (int it = 0; it < m; ++it) {
        if (lanczos) {
            const int vs = it % 3, ws = (it + 1) % 3, ps = (it + 2) % 3;
            // the pair runs as a programmatic dependent chain: each launch is
            // set up while the kernel before it runs (paper heat, 100^3,
            // 1600 short launches a query: 102.8 -> 100.5 ms).  The Arnoldi
            // chain below is launched plainly: its long multi-wave kernels
            // gained nothing and lost 1 % with it.
            {
                LaunchScope ls(p->ctx, "csr_spmv");
                KV_CHECK_CUDA(launch_dep(dep_launch_ok(p->ctx), k_spmv<T, true>, gv, dim3(CNT), 0, st, s->d_rp,
                                         s->d_col, (const T*)s->d_val, s->d_b, va, vs, ws, n, N, aug, stp, H, m, it,
                                         partials, counters, nbx));
            }
            {
                LaunchScope ls(p->ctx, "csr_lanczos_update");
                KV_CHECK_CUDA(launch_dep(dep_launch_ok(p->ctx), it == 0 ? k_lanczos3_update<T, true>
                                                                        : k_lanczos3_update<T, false>,
                                         gu, dim3(CNT), 0, st, va, ws, vs, ps, N, stp, H, P, cd, cinl, m, it,
                                         partials, counters, nbx));
            }
            const int rc = launch_project(p, j0, ncols, (T*)V + (int64_t)ws * N, va.cstride, it + 1);
            if (rc) return rc;
        } else {
            if (p->spmm_G != 0 && !(p->flags & KV_FLAG_NO_SPMM)) {
                // grouped SpMM: the matrix is read once per group of |spmm_G| columns
                LaunchScope ls(p->ctx, "csr_spmm");
                if (!spmm_dispatch<T>(p, p->spmm_G, p->spmm_LPR, va, it, it + 1, aug, stp, it, ncols, st)) {
                    set_error("no SpMM kernel for G=%d LPR=%d", p->spmm_G, p->spmm_LPR);
                    return KV_EINVAL;
                }
                KV_CHECK_CUDA(cudaGetLastError());
            } else {
                LaunchScope ls(p->ctx, "csr_spmv");
                k_spmv<T, false><<<gv, CNT, 0, st>>>(s->d_rp, s->d_col, (const T*)s->d_val, s->d_b, va, it, it + 1, n,
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
