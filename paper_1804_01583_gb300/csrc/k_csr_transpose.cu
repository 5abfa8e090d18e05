// k_csr_transpose.cu -- A^T of a CSR matrix on the device, for the transpose
// dynamics of Sec. 4.1 (x' = A^T x started at the rows of C), and the last
// row of A'^T = [[A^T, 0], [b^T, 0]] (b . x) for the augmented runs.
//
// Transpose: count the entries of every column (integer atomics), exclusive
// prefix sum into the new row pointers, scatter (column c's entries land in
// row c in atomic order), then sort every new row by its column index (the
// original row), so the result does not depend on the order of the atomics.
#include "kv_internal.h"
#include "reduce.cuh"

namespace kv {

constexpr int TNT = 256;
constexpr int SCAN_B = 1024;  // elements per scan block (TNT threads x 4)

__global__ void __launch_bounds__(TNT) k_ct_count(const int32_t* col, int64_t nnz, unsigned* cnt) {
    for (int64_t e = (int64_t)blockIdx.x * TNT + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * TNT)
        atomicAdd(&cnt[col[e]], 1u);
}

// exclusive scan of cnt[0..n) within blocks of SCAN_B; block totals to bsum
__global__ void __launch_bounds__(TNT) k_ct_scan_blocks(const unsigned* cnt, int64_t n, int64_t* out, int64_t* bsum) {
    __shared__ int64_t wsum[TNT / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * 4;
    int64_t v[4], run = 0;
    for (int q = 0; q < 4; ++q) {
        v[q] = base + q < n ? (int64_t)cnt[base + q] : 0;
        run += v[q];
    }
    // inclusive scan of the per-thread sums across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int64_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += wsum[w];
    int64_t acc = woff + inc - run;  // exclusive prefix of this thread's first element
    for (int q = 0; q < 4; ++q) {
        if (base + q < n) out[base + q] = acc;
        acc += v[q];
    }
    if (threadIdx.x == TNT - 1) bsum[blockIdx.x] = woff + inc;
}

// one block: exclusive scan of the block totals, in order
__global__ void __launch_bounds__(TNT) k_ct_scan_totals(int64_t* bsum, int64_t nb, int64_t* total) {
    __shared__ int64_t wsum[TNT / 32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c0 = 0; c0 < nb; c0 += TNT) {
        const int64_t i = c0 + threadIdx.x;
        const int64_t v = i < nb ? bsum[i] : 0;
        int64_t inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        int64_t woff = 0;
        for (int w = 0; w < warp; ++w) woff += wsum[w];
        const int64_t excl = carry + woff + inc - v;
        __syncthreads();
        if (i < nb) bsum[i] = excl;
        if (threadIdx.x == TNT - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(TNT) k_ct_scan_add(int64_t* out, int64_t n, const int64_t* bsum, unsigned long long* cursor) {
    for (int64_t i = (int64_t)blockIdx.x * TNT + threadIdx.x; i < n; i += (int64_t)gridDim.x * TNT) {
        const int64_t v = out[i] + bsum[i / SCAN_B];
        out[i] = v;
        cursor[i] = (unsigned long long)v;
    }
}

template <typename T>
__global__ void __launch_bounds__(TNT) k_ct_scatter(const int64_t* rp, const int32_t* col, const T* val, int64_t n,
                                                    unsigned long long* cursor, int32_t* colT, T* valT) {
    for (int64_t r = (int64_t)blockIdx.x * TNT + threadIdx.x; r < n; r += (int64_t)gridDim.x * TNT)
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
            const int64_t pos = (int64_t)atomicAdd(&cursor[col[e]], 1ULL);
            colT[pos] = (int32_t)r;
            valT[pos] = val[e];
        }
}

template <typename T>
__global__ void __launch_bounds__(TNT) k_ct_sort(const int64_t* rpT, int64_t n, int32_t* colT, T* valT) {
    for (int64_t r = (int64_t)blockIdx.x * TNT + threadIdx.x; r < n; r += (int64_t)gridDim.x * TNT) {
        const int64_t a = rpT[r], b = rpT[r + 1];
        for (int64_t i = a + 1; i < b; ++i) {  // insertion sort by column (rows of A^T are short)
            const int32_t c = colT[i];
            const T v = valT[i];
            int64_t q = i - 1;
            while (q >= a && colT[q] > c) {
                colT[q + 1] = colT[q];
                valT[q + 1] = valT[q];
                --q;
            }
            colT[q + 1] = c;
            valT[q + 1] = v;
        }
    }
}

int csr_build_transpose(Sys* s) {
    if (s->d_rpT) return KV_OK;
    Ctx* c = s->ctx;
    const int64_t n = s->n, nnz = s->nnz;
    const size_t es = s->val_prec == KV_FP32 ? 4 : 8;
    const int64_t nb = (n + SCAN_B - 1) / SCAN_B;
    int64_t* rpT = (int64_t*)c->arena.alloc((size_t)(n + 1) * 8);
    int32_t* colT = (int32_t*)c->arena.alloc((size_t)std::max<int64_t>(nnz, 1) * 4);
    void* valT = c->arena.alloc((size_t)std::max<int64_t>(nnz, 1) * es);
    unsigned* cnt = (unsigned*)c->arena.alloc((size_t)n * 4);
    int64_t* bsum = (int64_t*)c->arena.alloc((size_t)(nb + 1) * 8);
    unsigned long long* cursor = (unsigned long long*)c->arena.alloc((size_t)n * 8);
    auto release_scratch = [&]() {
        c->arena.free(cnt);
        c->arena.free(bsum);
        c->arena.free(cursor);
    };
    if (!rpT || !colT || !valT || !cnt || !bsum || !cursor) {
        release_scratch();
        c->arena.free(rpT);
        c->arena.free(colT);
        c->arena.free(valT);
        set_error("pool cannot hold the transposed matrix (%lld nnz)", (long long)nnz);
        return KV_ENOMEM;
    }
    cudaStream_t st = c->stream;
    const unsigned g = (unsigned)std::min<int64_t>((std::max<int64_t>(nnz, n) + TNT - 1) / TNT, 152 * 16);
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)n * 4, st);
    if (e == cudaSuccess) {
        k_ct_count<<<g, TNT, 0, st>>>(s->d_col, nnz, cnt);
        k_ct_scan_blocks<<<(unsigned)nb, TNT, 0, st>>>(cnt, n, rpT, bsum);
        k_ct_scan_totals<<<1, TNT, 0, st>>>(bsum, nb, rpT + n);
        k_ct_scan_add<<<g, TNT, 0, st>>>(rpT, n, bsum, cursor);
        if (es == 4) {
            k_ct_scatter<float><<<g, TNT, 0, st>>>(s->d_rp, s->d_col, (const float*)s->d_val, n, cursor, colT, (float*)valT);
            k_ct_sort<float><<<g, TNT, 0, st>>>(rpT, n, colT, (float*)valT);
        } else {
            k_ct_scatter<double><<<g, TNT, 0, st>>>(s->d_rp, s->d_col, (const double*)s->d_val, n, cursor, colT,
                                                   (double*)valT);
            k_ct_sort<double><<<g, TNT, 0, st>>>(rpT, n, colT, (double*)valT);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release_scratch();
    if (e != cudaSuccess) {
        c->arena.free(rpT);
        c->arena.free(colT);
        c->arena.free(valT);
        set_error("CSR transpose failed: %s", cudaGetErrorString(e));
        return KV_ECUDA;
    }
    s->d_rpT = rpT;
    s->d_colT = colT;
    s->d_valT = valT;
    return KV_OK;
}

// W[n] = s_j (b . X[0:n]) for every column of the run (blockIdx.y): the last
// row of A'^T, after the SpMV has written rows 0..n-1 (without b terms).
template <typename T>
__global__ void __launch_bounds__(TNT) k_row_dot(const double* __restrict__ b, const T* base, int64_t cstride,
                                                 int xslot, int wslot, int64_t n, int64_t N, const ColState* st,
                                                 int j, double* partials, unsigned* counters) {
    const int cidx = blockIdx.y;
    const ColState* s = st + cidx;
    if (s->done) return;
    const T* X = base + cidx * cstride + (int64_t)xslot * N;
    T* W = const_cast<T*>(base) + cidx * cstride + (int64_t)wslot * N;
    double acc = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * TNT + threadIdx.x; r < n; r += (int64_t)gridDim.x * TNT)
        acc = fma(b[r], (double)X[r], acc);
    __shared__ double sh[TNT / 32];
    __shared__ int flag;
    const double part = block_sum<TNT>(acc, sh);
    double* pc = partials + (int64_t)cidx * gridDim.x;
    if (!grid_arrive(part, pc, counters + cidx, blockIdx.x, gridDim.x, &flag)) return;
    const double tot = grid_finish<TNT>(pc, gridDim.x, counters + cidx, sh);
    if (threadIdx.x == 0) W[n] = (T)(s->s[j] * tot);
}

int row_dot_blocks() { return 152 * 2; }

int launch_row_dot(Prob* p, int j0, int ncols, void* V, int xslot, int wslot, int it) {
    LaunchScope ls(p->ctx, "row_dot");
    const dim3 grd((unsigned)row_dot_blocks(), (unsigned)ncols);
    const int64_t cstride = (int64_t)p->nvec * p->N;
    double* part = p->d_rowdot;
    unsigned* cnt = (unsigned*)(p->d_rowdot + (size_t)p->i * row_dot_blocks()) + j0;
    part += (size_t)j0 * row_dot_blocks();
    if (p->prec == KV_FP32)
        k_row_dot<float><<<grd, TNT, 0, p->ctx->stream>>>(p->d_brow, (const float*)V, cstride, xslot, wslot,
                                                          p->sys->n, p->N, p->d_state + j0, it, part, cnt);
    else
        k_row_dot<double><<<grd, TNT, 0, p->ctx->stream>>>(p->d_brow, (const double*)V, cstride, xslot, wslot,
                                                           p->sys->n, p->N, p->d_state + j0, it, part, cnt);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

// basis[j][r][k] = inner[r][j][k]: the runs of the transpose dynamics give the
// basis matrix one output row at a time
__global__ void __launch_bounds__(TNT) k_basis_transpose(const double* in, double* out, int R, int J, int64_t S) {
    const int64_t tot = (int64_t)R * J * S;
    for (int64_t e = (int64_t)blockIdx.x * TNT + threadIdx.x; e < tot; e += (int64_t)gridDim.x * TNT) {
        const int64_t k = e % S;
        const int64_t rj = e / S;
        const int64_t jj = rj % J, r = rj / J;
        out[(jj * R + r) * S + k] = in[e];
    }
}

int launch_basis_transpose(const Prob* inner, double* out, cudaStream_t st) {
    const int64_t S = inner->steps + 1;
    const int64_t tot = (int64_t)inner->i * inner->o * S;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tot + TNT - 1) / TNT, 152 * 8));
    k_basis_transpose<<<g, TNT, 0, st>>>(inner->d_basis, out, inner->i, inner->o, S);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

}  // namespace kv
