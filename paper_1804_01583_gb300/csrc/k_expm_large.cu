// k_expm_large.cu -- e^{t_k H} e_1 for Krylov dimensions above the
// shared-memory exponential's 64 (Eq. approx-formula, Sec. 4.2), in global
// memory with FP64 GEMMs.
//
// For one column with dimension k (known on the device only: the column's
// m_used, or a checkpoint dimension of the error control):
//   1. X = dt H_k, s = the smallest scaling with ||X / 2^s||_1 = r where the
//      Taylor remainder of degree 18, r^19 / 19! / (1 - r/20), is below 2^-53
//      (derived from the Lagrange remainder with the geometric tail bound);
//   2. E = T_18(X / 2^s) by Paterson-Stockmeyer (X^2, X^3, X^4, then Horner
//      in X^4 over blocks c_{4i} I + c_{4i+1} X + c_{4i+2} X^2 + c_{4i+3} X^3,
//      c_j = 1/j!), then s squarings: E = e^{dt H_k};
//   3. U[:, t] = e^{t dt H_k} e_1 for t = 0..steps by doubling: with
//      P_i = E^(2^i), U[:, 2^i + c] = P_i U[:, c] for c < 2^i, P_{i+1} = P_i^2
//      (ceil(log2(steps+1)) GEMM rounds instead of steps matrix-vector
//      products in sequence);
//   4. basis rows beta0 P U (o x (steps+1)) and the last row |U[k-1, :]|, the
//      integrand of the Lemma-1 bound.
// Every launch is sized for the largest dimension m and reads k from the
// column state; tiles beyond k return at once, and a checkpoint of a column
// that has stopped does nothing.  The number of squaring launches is fixed
// (SQ_LAUNCHES); those beyond the column's s copy instead, so the launch
// sequence does not depend on device data (it can be captured in a graph).
//
// This replaces the paper's Pade exponential (Sec. 4.1) above dimension 64:
// the same e^{t H} up to rounding, without a linear solve.
#include <math.h>

#include "kv_internal.h"

namespace kv {

constexpr int GT = 32;          // GEMM tile: GT x GT outputs per CTA
constexpr int GNT = 256;        // 16 x 16 threads, 2 x 2 outputs each
constexpr int SQ_LAUNCHES = 32; // squarings enqueued (even); handles ||dt H||_1 up to 2^32

struct KDim {
    const ColState* st;
    int dim;  // > 0: checkpoint dimension (columns that have stopped skip); 0: m_used
};

__device__ __forceinline__ int kdim(const KDim& d) {
    if (d.dim > 0) return d.st->done ? -1 : d.dim;
    return d.st->m_used;
}

struct Lin4 {  // c0 I + c1 X + c2 X2 + c3 X3 (leading dimension ld; X3 may be null)
    double c0, c1, c2, c3;
    const double *X, *X2, *X3;
    int ld;
};

struct GemmArgs {
    const double* A;
    int lda;
    const double* B;
    int ldb;
    double* C;
    int ldc;
    int M, N, K;      // fixed sizes; -1 = the column's k
    KDim kd;
    int epi;          // 0: C = AB; 1: C = AB + lin; 2: C = beta0 AB (beta0 of the column)
    Lin4 lin;
    const int* gate;  // squaring gate: q >= *gate -> C = A (copy)
    int q;
};

__device__ __forceinline__ double lin_at(const Lin4& l, int r, int c) {
    const int64_t e = (int64_t)r * l.ld + c;
    double v = (r == c) ? l.c0 : 0.0;
    v = fma(l.c1, l.X[e], v);
    v = fma(l.c2, l.X2[e], v);
    if (l.X3) v = fma(l.c3, l.X3[e], v);
    return v;
}

__global__ void __launch_bounds__(GNT) k_dgemm(GemmArgs g) {
    const int k = kdim(g.kd);
    if (k < 0) return;
    const int M = g.M < 0 ? k : g.M, N = g.N < 0 ? k : g.N, K = g.K < 0 ? k : g.K;
    const int r0 = blockIdx.y * GT, c0 = blockIdx.x * GT;
    if (r0 >= M || c0 >= N) return;
    if (k == 0) {  // zero column: zero outputs (basis rows)
        for (int e = threadIdx.x; e < GT * GT; e += GNT) {
            const int r = r0 + e / GT, c = c0 + e % GT;
            if (r < M && c < N) g.C[(int64_t)r * g.ldc + c] = 0.0;
        }
        return;
    }
    if (g.gate && g.q >= *g.gate) {
        for (int e = threadIdx.x; e < GT * GT; e += GNT) {
            const int r = r0 + e / GT, c = c0 + e % GT;
            if (r < M && c < N) g.C[(int64_t)r * g.ldc + c] = g.A[(int64_t)r * g.lda + c];
        }
        return;
    }
    __shared__ double As[GT][GT + 1], Bs[GT][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;
    for (int kk = 0; kk < K; kk += GT) {
        for (int e = threadIdx.x; e < GT * GT; e += GNT) {
            const int a = e / GT, b = e % GT;
            const int ar = r0 + a, ac = kk + b;
            As[a][b] = (ar < M && ac < K) ? g.A[(int64_t)ar * g.lda + ac] : 0.0;
            const int br = kk + a, bc = c0 + b;
            Bs[a][b] = (br < K && bc < N) ? g.B[(int64_t)br * g.ldb + bc] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int l = 0; l < GT; ++l) {
            const double a0 = As[2 * ty][l], a1 = As[2 * ty + 1][l];
            const double b0 = Bs[l][2 * tx], b1 = Bs[l][2 * tx + 1];
            acc00 = fma(a0, b0, acc00);
            acc01 = fma(a0, b1, acc01);
            acc10 = fma(a1, b0, acc10);
            acc11 = fma(a1, b1, acc11);
        }
        __syncthreads();
    }
    const double accs[2][2] = {{acc00, acc01}, {acc10, acc11}};
    const double beta0 = g.epi == 2 ? g.kd.st->beta0 : 1.0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const int r = r0 + 2 * ty + i, c = c0 + 2 * tx + jj;
            if (r >= M || c >= N) continue;
            double v = accs[i][jj];
            if (g.epi == 1) v += lin_at(g.lin, r, c);
            if (g.epi == 2) v *= beta0;
            g.C[(int64_t)r * g.ldc + c] = v;
        }
}

// C = lin on the leading k x k block
__global__ void __launch_bounds__(GNT) k_lincomb(double* C, int ldc, Lin4 lin, KDim kd) {
    const int k = kdim(kd);
    if (k <= 0) return;
    const int64_t kk = (int64_t)k * k;
    for (int64_t e = (int64_t)blockIdx.x * GNT + threadIdx.x; e < kk; e += (int64_t)gridDim.x * GNT) {
        const int r = (int)(e / k), c = (int)(e - (int64_t)r * k);
        C[(int64_t)r * ldc + c] = lin_at(lin, r, c);
    }
}

// X = dt H_k (leading k x k block of the column's (m+1) x m H)
__global__ void __launch_bounds__(GNT) k_lx_load(const double* H, int ldh, double* X, int ldx, double dt, KDim kd) {
    const int k = kdim(kd);
    if (k <= 0) return;
    const int64_t kk = (int64_t)k * k;
    for (int64_t e = (int64_t)blockIdx.x * GNT + threadIdx.x; e < kk; e += (int64_t)gridDim.x * GNT) {
        const int r = (int)(e / k), c = (int)(e - (int64_t)r * k);
        X[(int64_t)r * ldx + c] = dt * H[(int64_t)r * ldh + c];
    }
}

// column sums of |X|, one warp per column
__global__ void __launch_bounds__(GNT) k_lx_colsum(const double* X, int ldx, double* cs, KDim kd) {
    const int k = kdim(kd);
    if (k <= 0) return;
    const int lane = threadIdx.x & 31;
    for (int c = blockIdx.x * (GNT / 32) + (threadIdx.x >> 5); c < k; c += gridDim.x * (GNT / 32)) {
        double s = 0.0;
        for (int r = lane; r < k; r += 32) s += fabs(X[(int64_t)r * ldx + c]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) cs[c] = s;
    }
}

// one CTA: ||X||_1, the scaling s (device int, at most smax) and 2^-s
__global__ void __launch_bounds__(GNT) k_lx_scaling(const double* cs, int* nsq, double* scale, int smax, KDim kd) {
    __shared__ double red[GNT / 32];
    const int k = kdim(kd);
    if (k <= 0) return;
    double mx = 0.0;
    for (int c = threadIdx.x; c < k; c += GNT) mx = fmax(mx, cs[c]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double nrm = 0.0;
    for (int w = 0; w < GNT / 32; ++w) nrm = fmax(nrm, red[w]);
    // Taylor degree 18: remainder <= r^19 / 19! * 1 / (1 - r/20) for r < 20
    const double inv_fact19 = 1.0 / 121645100408832000.0;  // 19! is exactly representable
    int s = 0;
    double r = nrm;
    while (s < smax) {
        double p = 1.0;
        for (int e = 0; e < 19; ++e) p *= r;
        if (r < 20.0 && p * inv_fact19 / (1.0 - r / 20.0) <= 0x1p-53) break;
        r *= 0.5;
        ++s;
    }
    *nsq = s;
    *scale = ldexp(1.0, -s);
}

__global__ void __launch_bounds__(GNT) k_lx_scale(double* X, int ldx, const double* scale, KDim kd) {
    const int k = kdim(kd);
    if (k <= 0) return;
    const double f = *scale;
    const int64_t kk = (int64_t)k * k;
    for (int64_t e = (int64_t)blockIdx.x * GNT + threadIdx.x; e < kk; e += (int64_t)gridDim.x * GNT) {
        const int r = (int)(e / k), c = (int)(e - (int64_t)r * k);
        X[(int64_t)r * ldx + c] *= f;
    }
}

// U[:, 0] = e_1
__global__ void __launch_bounds__(GNT) k_lx_init_u(double* U, int ldu, KDim kd) {
    const int k = kdim(kd);
    if (k <= 0) return;
    for (int r = blockIdx.x * GNT + threadIdx.x; r < k; r += gridDim.x * GNT) U[(int64_t)r * ldu] = (r == 0) ? 1.0 : 0.0;
}

// hl[t] = |U[k-1, t]| (0 for a zero column)
__global__ void __launch_bounds__(GNT) k_lx_hlast(const double* U, int ldu, int S, double* hl, KDim kd) {
    const int k = kdim(kd);
    if (k < 0) return;
    for (int t = blockIdx.x * GNT + threadIdx.x; t < S; t += gridDim.x * GNT)
        hl[t] = k == 0 ? 0.0 : fabs(U[(int64_t)(k - 1) * ldu + t]);
}

// ---------------------------------------------------------------- host side
size_t large_expm_scratch_doubles(int m, int steps) {
    return (size_t)6 * m * m + (size_t)m * (steps + 1) + (size_t)m + 64;
}

static int gemm(Prob* p, const double* A, int lda, const double* B, int ldb, double* C, int ldc, int M, int N, int K,
                KDim kd, int epi = 0, Lin4 lin = Lin4{}, const int* gate = nullptr, int q = 0) {
    const int Mx = M < 0 ? p->m : M, Nx = N < 0 ? p->m : N;
    dim3 grd((unsigned)((Nx + GT - 1) / GT), (unsigned)((Mx + GT - 1) / GT));
    GemmArgs g{A, lda, B, ldb, C, ldc, M, N, K, kd, epi, lin, gate, q};
    k_dgemm<<<grd, GNT, 0, p->ctx->stream>>>(g);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

// e^{t dt H_k} e_1 for t = 0..steps of column j at dimension dim (0: m_used),
// the integrand row into hlast, and (write_basis) the basis rows.
int launch_expm_large_column(Prob* p, int j, int dim, bool write_basis) {
    const int m = p->m, S = p->steps + 1;
    cudaStream_t st = p->ctx->stream;
    LaunchScope ls(p->ctx, dim > 0 ? "error_expm" : "expm_large");
    const KDim kd{p->d_state + j, dim};
    double* X = p->d_lx;
    double* X2 = X + (size_t)m * m;
    double* X3 = X2 + (size_t)m * m;
    double* X4 = X3 + (size_t)m * m;
    double* T0 = X4 + (size_t)m * m;
    double* T1 = T0 + (size_t)m * m;
    double* U = T1 + (size_t)m * m;
    double* cs = U + (size_t)m * S;
    double* scale = cs + m;
    int* nsq = (int*)(scale + 8);
    const unsigned eb = (unsigned)std::min<int64_t>(((int64_t)m * m + GNT - 1) / GNT, 152 * 8);
    const double* H = p->d_H + (int64_t)j * (m + 1) * m;
    k_lx_load<<<eb, GNT, 0, st>>>(H, m, X, m, p->dt, kd);
    k_lx_colsum<<<(unsigned)((m + 7) / 8), GNT, 0, st>>>(X, m, cs, kd);
    k_lx_scaling<<<1, GNT, 0, st>>>(cs, nsq, scale, SQ_LAUNCHES, kd);
    k_lx_scale<<<eb, GNT, 0, st>>>(X, m, scale, kd);
    KV_CHECK_CUDA(cudaGetLastError());
    int rc = gemm(p, X, m, X, m, X2, m, -1, -1, -1, kd);
    if (!rc) rc = gemm(p, X2, m, X, m, X3, m, -1, -1, -1, kd);
    if (!rc) rc = gemm(p, X2, m, X2, m, X4, m, -1, -1, -1, kd);
    if (rc) return rc;
    // Paterson-Stockmeyer: blocks B_i = c_{4i} I + c_{4i+1} X + c_{4i+2} X^2 + c_{4i+3} X^3
    double c[19];
    c[0] = 1.0;
    for (int i = 1; i <= 18; ++i) c[i] = c[i - 1] / (double)i;
    auto blk = [&](int i) {
        return Lin4{c[4 * i], c[4 * i + 1], c[4 * i + 2], 4 * i + 3 <= 18 ? c[4 * i + 3] : 0.0, X, X2,
                    4 * i + 3 <= 18 ? X3 : nullptr, m};
    };
    k_lincomb<<<eb, GNT, 0, st>>>(T0, m, blk(4), kd);  // B_4 = c16 I + c17 X + c18 X^2
    KV_CHECK_CUDA(cudaGetLastError());
    double* cur = T0;
    double* nxt = T1;
    for (int i = 3; i >= 0; --i) {  // T = T X^4 + B_i
        rc = gemm(p, cur, m, X4, m, nxt, m, -1, -1, -1, kd, 1, blk(i));
        if (rc) return rc;
        std::swap(cur, nxt);
    }
    // squarings (SQ_LAUNCHES is even: the result ends in `cur`)
    for (int q = 0; q < SQ_LAUNCHES; ++q) {
        rc = gemm(p, cur, m, cur, m, nxt, m, -1, -1, -1, kd, 0, Lin4{}, nsq, q);
        if (rc) return rc;
        std::swap(cur, nxt);
    }
    // doubling over the output steps: P_0 = E (in cur), spare buffers X2 / X3
    k_lx_init_u<<<(unsigned)((m + GNT - 1) / GNT), GNT, 0, st>>>(U, S, kd);
    KV_CHECK_CUDA(cudaGetLastError());
    const double* P = cur;
    double* spare[2] = {X2, X3};
    int sp = 0;
    for (int off = 1; off < S; off *= 2) {
        const int len = std::min(off, S - off);
        rc = gemm(p, P, m, U, S, U + off, S, -1, len, -1, kd);
        if (rc) return rc;
        if (2 * off < S) {
            rc = gemm(p, P, m, P, m, spare[sp], m, -1, -1, -1, kd);
            if (rc) return rc;
            P = spare[sp];
            sp ^= 1;
        }
    }
    k_lx_hlast<<<(unsigned)((S + GNT - 1) / GNT), GNT, 0, st>>>(U, S, S, p->d_hlast + (int64_t)j * S, kd);
    KV_CHECK_CUDA(cudaGetLastError());
    if (write_basis) {
        rc = gemm(p, p->d_P + (int64_t)j * p->o * m, m, U, S, p->d_basis + (int64_t)j * p->o * S, S, p->o, S, -1, kd,
                  2);
        if (rc) return rc;
    }
    return KV_OK;
}

}  // namespace kv
