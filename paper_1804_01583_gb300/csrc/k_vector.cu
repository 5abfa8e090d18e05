// k_vector.cu -- initial Krylov vector for sparse and dense columns.
//
// The column E_j (with the constant-1 entry appended when the column carries
// the constant variable, Sec. 2.1) is written into the first Krylov buffer
// unnormalised; k_init_norm reduces ||E_j||^2 deterministically and its last
// block sets beta0, the read scale s[0] = 1/beta0 and P[:, 0] = C v_0.
#include "kv_internal.h"
#include "reduce.cuh"

namespace kv {

constexpr int VNT = 256;

template <typename T>
__global__ void k_scatter(T* __restrict__ B, const int64_t* __restrict__ idx, const double* __restrict__ val,
                          int64_t nnz, int64_t N, int* status) {
    for (int64_t e = (int64_t)blockIdx.x * VNT + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * VNT) {
#ifdef KV_DEBUG
        // debug build: an index outside the vector is skipped, not written
        if (idx[e] < 0 || idx[e] >= N) {
            atomicOr(status, KV_ST_INDEX);
            continue;
        }
#endif
        B[idx[e]] = (T)val[e];
    }
}

template <typename T>
__global__ void k_convert(T* __restrict__ B, const double* __restrict__ src, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * VNT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VNT)
        B[e] = (T)src[e];
}

template <typename T>
__global__ void __launch_bounds__(VNT) k_init_norm(const T* __restrict__ B, int64_t N, ColState* st, double* P,
                                                   CDesc cd, int m, Reduce red) {
    __shared__ double sh[VNT / 32];
    __shared__ int flag;
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * VNT + threadIdx.x; e < N; e += (int64_t)gridDim.x * VNT) {
        const double v = (double)B[e];
        acc = fma(v, v, acc);
    }
    const double part = block_sum<VNT>(acc, sh);
    if (!grid_arrive(part, red.partials, red.counter, blockIdx.x, gridDim.x, &flag)) return;
    const double tot = grid_finish<VNT>(red.partials, gridDim.x, red.counter, sh);
    __shared__ double s0;
    if (threadIdx.x == 0) {
        const double b0 = sqrt(tot);
        st->beta0 = b0;
        st->m_used = m;
        st->status = isfinite(b0) ? 0 : KV_ST_NONFINITE;
        if (!(b0 > 0.0) || !isfinite(b0)) {
            st->done = 1;
            st->m_used = 0;
            s0 = 0.0;
        } else {
            st->done = 0;
            st->s[0] = 1.0 / b0;
            s0 = 1.0 / b0;
        }
    }
    __syncthreads();
    if (cd.o > PROJ_INLINE_MAX) return;  // launch_project takes the rows
    for (int r = 0; r < cd.o; ++r) {
        double v = 0.0;
        for (int64_t e = cd.rp[r] + threadIdx.x; e < cd.rp[r + 1]; e += VNT)
            v += c_entry(cd, e, B, &st->status);
        v = block_sum<VNT>(v, sh);
        if (threadIdx.x == 0) P[(int64_t)r * m] = s0 * v;
    }
}

// P[r][jcol] = s_jcol (C_r . w) for every row of C, one warp per row, for the
// columns of a launch group (blockIdx.y); a column that stopped before jcol
// is skipped (its P columns past m_used are not used)
template <typename T>
__global__ void __launch_bounds__(VNT) k_project(const T* w0, int64_t cstride, ColState* st, CDesc cd,
                                                 double* P0, int64_t pstride, int m, int jcol) {
    const int c = blockIdx.y;
    ColState* s = st + c;
    if (s->done && s->m_used <= jcol) return;
    const T* W = w0 + c * cstride;
    double* P = P0 + c * pstride;
    const double sc = s->s[jcol];
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (VNT / 32);
    for (int64_t r = (int64_t)blockIdx.x * (VNT / 32) + (threadIdx.x >> 5); r < cd.o; r += nw) {
        double v = 0.0;
        for (int64_t e = cd.rp[r] + lane; e < cd.rp[r + 1]; e += 32) v += c_entry(cd, e, W, &s->status);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) P[r * m + jcol] = sc * v;
    }
}

int launch_project(Prob* p, int j0, int ncols, const void* w0, int64_t cstride, int jcol) {
    if (p->o <= PROJ_INLINE_MAX || jcol >= p->m) return KV_OK;
    LaunchScope ls(p->ctx, "project");
    CDesc cd{p->o, p->d_crp, p->d_ccol, p->d_cval, p->N};
    int64_t g = ((int64_t)p->o + (VNT / 32) - 1) / (VNT / 32);
    if (g > 152 * 16) g = 152 * 16;
    const dim3 grd((unsigned)g, (unsigned)ncols);
    double* P0 = p->d_P + (int64_t)j0 * p->o * p->m;
    const int64_t ps = (int64_t)p->o * p->m;
    if (p->prec == KV_FP32)
        k_project<float><<<grd, VNT, 0, p->ctx->stream>>>((const float*)w0, cstride, p->d_state + j0, cd, P0, ps,
                                                          p->m, jcol);
    else
        k_project<double><<<grd, VNT, 0, p->ctx->stream>>>((const double*)w0, cstride, p->d_state + j0, cd, P0, ps,
                                                           p->m, jcol);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

static int grid_for(int64_t n) {
    int64_t b = (n + VNT - 1) / VNT;
    if (b > 152 * 8) b = 152 * 8;
    return (int)(b < 1 ? 1 : b);
}

int launch_scatter(Prob* p, int j, void* B) {
    const size_t es = elem_size(p->prec);
    KV_CHECK_CUDA(cudaMemsetAsync(B, 0, (size_t)p->N * es, p->ctx->stream));
    const int64_t nnz = p->sidx_n[j];  // exactly what kv_problem uploaded
    if (nnz == 0) return KV_OK;
    LaunchScope ls(p->ctx, "scatter");
    if (p->prec == KV_FP32)
        k_scatter<float><<<grid_for(nnz), VNT, 0, p->ctx->stream>>>((float*)B, p->d_sidx[j], p->d_sval[j], nnz, p->N,
                                                                    &p->d_state[j].status);
    else
        k_scatter<double><<<grid_for(nnz), VNT, 0, p->ctx->stream>>>((double*)B, p->d_sidx[j], p->d_sval[j], nnz,
                                                                     p->N, &p->d_state[j].status);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

int launch_dense_to(Prob* p, int j, void* B) {
    LaunchScope ls(p->ctx, "dense_init");
    if (p->prec == KV_FP32)
        k_convert<float><<<grid_for(p->N), VNT, 0, p->ctx->stream>>>((float*)B, p->d_dense[j], p->N);
    else
        k_convert<double><<<grid_for(p->N), VNT, 0, p->ctx->stream>>>((double*)B, p->d_dense[j], p->N);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

int launch_init_norm(Prob* p, int j, void* B) {
    {
        LaunchScope ls(p->ctx, "init_norm");
        const int g = grid_for(p->N);
        CDesc cd{p->o, p->d_crp, p->d_ccol, p->d_cval, p->N};
        ColState* st = p->d_state + j;
        double* P = p->d_P + (int64_t)j * p->o * p->m;
        if (p->prec == KV_FP32)
            k_init_norm<float><<<g, VNT, 0, p->ctx->stream>>>((const float*)B, p->N, st, P, cd, p->m, p->red);
        else
            k_init_norm<double><<<g, VNT, 0, p->ctx->stream>>>((const double*)B, p->N, st, P, cd, p->m, p->red);
        KV_CHECK_CUDA(cudaGetLastError());
    }
    return launch_project(p, j, 1, B, 0, 0);
}

}  // namespace kv
