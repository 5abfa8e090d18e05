// k_expm_large.cu -- e^{t_k H} e_1 for all output steps in global memory
// with FP64 GEMMs (Eq. approx-formula, Sec. 4.2): the exponential of Krylov
// dimensions above the shared-memory kernels' 64, and the PROPAGATE schedule
// (u_k = M^k e_1, M = e^{dt H}) at every dimension, where it replaces s
// sequential matrix-vector products by ceil(log2(s+1)) rounds of GEMMs.
// Runs are batched: blockIdx.z selects the run, every buffer has a per-run
// stride.
//
// For one run with dimension k (known on the device only: the run's m_used,
// or a checkpoint dimension of the error control):
//   1. X = dt H_k, s = the smallest scaling with ||X / 2^s||_1 = r where the
//      Taylor remainder of degree 18, r^19 / 19! / (1 - r/20), is below 2^-53
//      (derived from the Lagrange remainder with the geometric tail bound);
//   2. E = T_18(X / 2^s) by Paterson-Stockmeyer (X^2, X^3, X^4, then Horner
//      in X^4 over blocks c_{4i} I + c_{4i+1} X + c_{4i+2} X^2 + c_{4i+3} X^3,
//      c_j = 1/j!), then s squarings: E = e^{dt H_k};
//   3. U[:, t] = e^{t dt H_k} e_1 for t = 0..steps by doubling: with
//      P_i = E^(2^i), U[:, 2^i + c] = P_i U[:, c] for c < 2^i, P_{i+1} = P_i^2;
//   4. basis rows beta0 P U (o x (steps+1)) and the last row |U[k-1, :]|, the
//      integrand of the Lemma-1 bound.
// Every launch is sized for the largest dimension m (for the checkpoint's
// dimension at a checkpoint) and reads k from the run's state; tiles beyond k
// return at once, and a checkpoint of a run that has stopped does nothing.
// Products with at most 16 rows or columns (the first doubling stages, the
// basis rows) run one thread per entry (k_dgemm_thin).  The Lanczos H is
// tridiagonal and the Arnoldi H upper Hessenberg, so the Taylor products and
// the first squarings are banded: each product is told the bands of its
// operands (entries outside them are exact zeros) and its tiles skip the
// K-tiles outside both, which only leaves out exact zero terms.  The number of
// squaring launches is fixed (SQ_LAUNCHES); those beyond the run's s return
// at once, the last one moving the result into the buffer the host reads
// when s is odd, so the launch sequence does not depend on device data (it
// can be captured in a graph).
//
// This is a different exponential from the paper's Pade (Sec. 4.1): the
// same e^{t H} up to rounding, without a linear solve.
#include <math.h>

#include <algorithm>

#include "kv_internal.h"

namespace kv {

constexpr int GT = 32;          // GEMM tile: GT x GT outputs per CTA
constexpr int GNT = 256;        // 16 x 16 threads, 2 x 2 outputs each
constexpr int SQ_LAUNCHES = 32; // squarings enqueued (even); handles ||dt H||_1 up to 2^32

// A(r, c) may be nonzero only for r - lo <= c <= r + up (BAND_DENSE: no band)
constexpr int BAND_DENSE = 1 << 28;
struct Band {
    int lo, up;
};
__host__ __device__ constexpr Band dense_band() { return Band{BAND_DENSE, BAND_DENSE}; }
static Band band_sum(Band a, Band b) {  // band of a product
    return Band{std::min(a.lo + b.lo, BAND_DENSE), std::min(a.up + b.up, BAND_DENSE)};
}
static Band band_max(Band a, Band b) { return Band{std::max(a.lo, b.lo), std::max(a.up, b.up)}; }

struct KDim {
    const ColState* st;  // the batch's first run; run z is st + z
    int dim;             // > 0: checkpoint dimension (runs that have stopped skip); 0: m_used
};

__device__ __forceinline__ int kdim(const KDim& d, int z) {
    const ColState* s = d.st + z;
    if (d.dim > 0) return s->done ? -1 : d.dim;
    return s->m_used;
}

struct Lin4 {  // c0 I + c1 X + c2 X2 + c3 X3 (leading dimension ld, run stride sz; X3 may be null)
    double c0, c1, c2, c3;
    const double *X, *X2, *X3;
    int ld;
    int64_t sz;
};

struct GemmArgs {
    const double* A;
    int lda;
    int64_t sA;
    const double* B;
    int ldb;
    int64_t sB;
    double* C;
    int ldc;
    int64_t sC;
    int M, N, K;      // fixed sizes; -1 = the run's k
    KDim kd;
    int epi;          // 0: C = AB; 1: C = AB + lin; 2: C = beta0 AB (beta0 of the run)
    Lin4 lin;
    const double* gate;  // squaring gate (per run, stride sG): launches q >= gate do not square
    int64_t sG;
    int q;
    Band ba, bb;      // bands of A and B
    int qlast;        // the last squaring launch (it moves the result when s is odd)
};

__device__ __forceinline__ double lin_at(const Lin4& l, int z, int r, int c) {
    const int64_t e = (int64_t)z * l.sz + (int64_t)r * l.ld + c;
    double v = (r == c) ? l.c0 : 0.0;
    v = fma(l.c1, l.X[e], v);
    v = fma(l.c2, l.X2[e], v);
    if (l.X3) v = fma(l.c3, l.X3[e], v);
    return v;
}

template <int TL>
__global__ void __launch_bounds__(GNT) k_dgemm(GemmArgs g) {
    constexpr int O = TL / 16;  // outputs per thread along each axis (16 x 16 threads)
    const int z = blockIdx.z;
    const int k = kdim(g.kd, z);
    if (k < 0) return;
    const int M = g.M < 0 ? k : g.M, N = g.N < 0 ? k : g.N, K = g.K < 0 ? k : g.K;
    const int r0 = blockIdx.y * TL, c0 = blockIdx.x * TL;
    if (r0 >= M || c0 >= N) return;
    const double* A = g.A + z * g.sA;
    const double* B = g.B + z * g.sB;
    double* C = g.C + z * g.sC;
    if (k == 0) {  // zero run: zero outputs (basis rows)
        for (int e = threadIdx.x; e < TL * TL; e += GNT) {
            const int r = r0 + e / TL, c = c0 + e % TL;
            if (r < M && c < N) C[(int64_t)r * g.ldc + c] = 0.0;
        }
        return;
    }
    if (g.gate) {
        const int s = (int)g.gate[z * g.sG];
        if (g.q >= s) {
            // the run's s squarings are done: the result stays in the buffer the
            // last one wrote, and only the last launch moves it to the buffer the
            // host reads next (the launch count is even: needed when s is odd)
            if (g.q == g.qlast && ((g.q - s) & 1) == 0) {
                for (int e = threadIdx.x; e < TL * TL; e += GNT) {
                    const int r = r0 + e / TL, c = c0 + e % TL;
                    if (r < M && c < N) C[(int64_t)r * g.ldc + c] = A[(int64_t)r * g.lda + c];
                }
            }
            return;
        }
    }
    __shared__ double As[TL][TL + 1], Bs[TL][TL + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[O][O];
#pragma unroll
    for (int i = 0; i < O; ++i)
#pragma unroll
        for (int jj = 0; jj < O; ++jj) acc[i][jj] = 0.0;
    // the inner indices l where both A(r0.., l) and B(l, c0..) may be nonzero
    const int l_lo = max(0, max(r0 - g.ba.lo, c0 - g.bb.up));
    const int l_hi = min(K - 1, min(r0 + TL - 1 + g.ba.up, c0 + TL - 1 + g.bb.lo));
    for (int kk = (l_lo / TL) * TL; kk <= l_hi; kk += TL) {
        for (int e = threadIdx.x; e < TL * TL; e += GNT) {
            const int a = e / TL, b = e % TL;
            const int ar = r0 + a, ac = kk + b;
            As[a][b] = (ar < M && ac < K) ? A[(int64_t)ar * g.lda + ac] : 0.0;
            const int br = kk + a, bc = c0 + b;
            Bs[a][b] = (br < K && bc < N) ? B[(int64_t)br * g.ldb + bc] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int l = 0; l < TL; ++l) {
            double av[O], bv[O];
#pragma unroll
            for (int i = 0; i < O; ++i) {
                av[i] = As[O * ty + i][l];
                bv[i] = Bs[l][O * tx + i];
            }
#pragma unroll
            for (int i = 0; i < O; ++i)
#pragma unroll
                for (int jj = 0; jj < O; ++jj) acc[i][jj] = fma(av[i], bv[jj], acc[i][jj]);
        }
        __syncthreads();
    }
    const double beta0 = g.epi == 2 ? (g.kd.st + z)->beta0 : 1.0;
#pragma unroll
    for (int i = 0; i < O; ++i)
#pragma unroll
        for (int jj = 0; jj < O; ++jj) {
            const int r = r0 + O * ty + i, c = c0 + O * tx + jj;
            if (r >= M || c >= N) continue;
            double v = acc[i][jj];
            if (g.epi == 1) v += lin_at(g.lin, z, r, c);
            if (g.epi == 2) v *= beta0;
            C[(int64_t)r * g.ldc + c] = v;
        }
}

// C = lin on the leading k x k block of each run
__global__ void __launch_bounds__(GNT) k_lincomb(double* C, int ldc, int64_t sC, Lin4 lin, KDim kd) {
    const int z = blockIdx.z;
    const int k = kdim(kd, z);
    if (k <= 0) return;
    const int64_t kk = (int64_t)k * k;
    for (int64_t e = (int64_t)blockIdx.x * GNT + threadIdx.x; e < kk; e += (int64_t)gridDim.x * GNT) {
        const int r = (int)(e / k), c = (int)(e - (int64_t)r * k);
        C[z * sC + (int64_t)r * ldc + c] = lin_at(lin, z, r, c);
    }
}

// X = dt H_k (leading k x k block of the run's (m+1) x m H)
__global__ void __launch_bounds__(GNT) k_lx_load(const double* H, int ldh, int64_t sH, double* X, int ldx, int64_t sX,
                                                 double dt, KDim kd) {
    const int z = blockIdx.z;
    const int k = kdim(kd, z);
    if (k <= 0) return;
    const int64_t kk = (int64_t)k * k;
    for (int64_t e = (int64_t)blockIdx.x * GNT + threadIdx.x; e < kk; e += (int64_t)gridDim.x * GNT) {
        const int r = (int)(e / k), c = (int)(e - (int64_t)r * k);
        X[z * sX + (int64_t)r * ldx + c] = dt * H[z * sH + (int64_t)r * ldh + c];
    }
}

// column sums of |X|, one warp per column
__global__ void __launch_bounds__(GNT) k_lx_colsum(const double* X, int ldx, int64_t sX, double* cs, int64_t sC,
                                                   KDim kd) {
    const int z = blockIdx.z;
    const int k = kdim(kd, z);
    if (k <= 0) return;
    const int lane = threadIdx.x & 31;
    for (int c = blockIdx.x * (GNT / 32) + (threadIdx.x >> 5); c < k; c += gridDim.x * (GNT / 32)) {
        double s = 0.0;
        for (int r = lane; r < k; r += 32) s += fabs(X[z * sX + (int64_t)r * ldx + c]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) cs[z * sC + c] = s;
    }
}

// one CTA per run: ||X||_1, the scaling s (stored as a double, at most smax)
// and 2^-s, next to the column sums
__global__ void __launch_bounds__(GNT) k_lx_scaling(const double* cs, int64_t sC, int m, int smax, KDim kd) {
    __shared__ double red[GNT / 32];
    const int z = blockIdx.z;
    const int k = kdim(kd, z);
    if (k <= 0) return;
    const double* c = cs + z * sC;
    double mx = 0.0;
    for (int q = threadIdx.x; q < k; q += GNT) mx = fmax(mx, c[q]);
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
    bool met = false;
    while (true) {
        double p = 1.0;
        for (int e = 0; e < 19; ++e) p *= r;
        if (r < 20.0 && p * inv_fact19 / (1.0 - r / 20.0) <= 0x1p-53) {
            met = true;
            break;
        }
        if (s == smax) break;
        r *= 0.5;
        ++s;
    }
    // more squarings needed than launched (a norm bound that did not hold, or
    // a norm beyond 2^32): reported, not truncated silently
    if (!met) atomicOr(&const_cast<ColState*>(kd.st + z)->status, KV_ST_SCALING);
    double* out = const_cast<double*>(c) + m;
    out[0] = (double)s;      // the squaring gate
    out[1] = ldexp(1.0, -s);  // the scale
}

__global__ void __launch_bounds__(GNT) k_lx_scale(double* X, int ldx, int64_t sX, const double* scale, int64_t sS,
                                                  KDim kd) {
    const int z = blockIdx.z;
    const int k = kdim(kd, z);
    if (k <= 0) return;
    const double f = scale[z * sS];
    const int64_t kk = (int64_t)k * k;
    for (int64_t e = (int64_t)blockIdx.x * GNT + threadIdx.x; e < kk; e += (int64_t)gridDim.x * GNT) {
        const int r = (int)(e / k), c = (int)(e - (int64_t)r * k);
        X[z * sX + (int64_t)r * ldx + c] *= f;
    }
}

// U[:, 0] = e_1
__global__ void __launch_bounds__(GNT) k_lx_init_u(double* U, int ldu, int64_t sU, KDim kd) {
    const int z = blockIdx.z;
    const int k = kdim(kd, z);
    if (k <= 0) return;
    for (int r = blockIdx.x * GNT + threadIdx.x; r < k; r += gridDim.x * GNT)
        U[z * sU + (int64_t)r * ldu] = (r == 0) ? 1.0 : 0.0;
}

// hl[t] = |U[k-1, t]| (0 for a zero run)
__global__ void __launch_bounds__(GNT) k_lx_hlast(const double* U, int ldu, int64_t sU, int S, double* hl, KDim kd) {
    const int z = blockIdx.z;
    const int k = kdim(kd, z);
    if (k < 0) return;
    for (int t = blockIdx.x * GNT + threadIdx.x; t < S; t += gridDim.x * GNT)
        hl[(int64_t)z * S + t] = k == 0 ? 0.0 : fabs(U[z * sU + (int64_t)(k - 1) * ldu + t]);
}

// ---------------------------------------------------------------- host side
// per-run scratch: X, X^2, X^3, X^4, two Horner / squaring buffers (m x m
// each), U (m x (steps+1)), the column sums (m) and the gate and scale
size_t large_expm_scratch_doubles(int m, int steps) {
    return (size_t)6 * m * m + (size_t)m * (steps + 1) + (size_t)m + 64;
}

// runs processed per batch: the scratch of one batch stays under 1 GB (at
// least one run)
int large_expm_batch(int m, int steps, int runs) {
    const size_t per = large_expm_scratch_doubles(m, steps) * 8;
    const size_t cap = (size_t)1 << 30;
    int64_t b = (int64_t)(cap / per);
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, runs);
}

// Thin products (M or N at most 16: the first doubling stages and the basis
// rows): one thread per output entry, four interleaved partial sums over K
// added in a fixed order.  The 32 x 32 tiles of k_dgemm would spend almost
// all of their FP64 work on zero padding there.  blockIdx.y = run.
__global__ void __launch_bounds__(GNT) k_dgemm_thin(GemmArgs g) {
    const int z = blockIdx.y;
    const int k = kdim(g.kd, z);
    if (k < 0) return;
    const int M = g.M < 0 ? k : g.M, N = g.N < 0 ? k : g.N, K = g.K < 0 ? k : g.K;
    const double* A = g.A + z * g.sA;
    const double* B = g.B + z * g.sB;
    double* C = g.C + z * g.sC;
    const double beta0 = g.epi == 2 ? (g.kd.st + z)->beta0 : 1.0;
    for (int64_t e = (int64_t)blockIdx.x * GNT + threadIdx.x; e < (int64_t)M * N; e += (int64_t)gridDim.x * GNT) {
        const int r = (int)(e / N), c = (int)(e - (int64_t)r * N);
        const double* a = A + (int64_t)r * g.lda;
        const double* b = B + c;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int kk = 0;
        for (; kk + 4 <= K; kk += 4) {
            s0 = fma(a[kk], b[(int64_t)kk * g.ldb], s0);
            s1 = fma(a[kk + 1], b[(int64_t)(kk + 1) * g.ldb], s1);
            s2 = fma(a[kk + 2], b[(int64_t)(kk + 2) * g.ldb], s2);
            s3 = fma(a[kk + 3], b[(int64_t)(kk + 3) * g.ldb], s3);
        }
        for (; kk < K; ++kk) s0 = fma(a[kk], b[(int64_t)kk * g.ldb], s0);
        C[(int64_t)r * g.ldc + c] = ((s0 + s1) + (s2 + s3)) * beta0;  // k == 0: K = 0, zero rows
    }
}

// The FP64 pipe of an SM is shared by its resident CTAs, so a product takes
// about (CTAs on the busiest SM) x (work of one CTA): ceil(tiles / SMs) x
// tile^2 (times K, the same for both tile sizes).
static int64_t waves_x_work(int M, int N, int nb, int tl) {
    const int64_t tiles = (int64_t)((N + tl - 1) / tl) * ((M + tl - 1) / tl) * nb;
    return (tiles + 151) / 152 * tl * tl;
}

static int gemm(Prob* p, int nb, const double* A, int lda, int64_t sA, const double* B, int ldb, int64_t sB, double* C,
                int ldc, int64_t sC, int M, int N, int K, KDim kd, int epi = 0, Lin4 lin = Lin4{},
                const double* gate = nullptr, int64_t sG = 0, int q = 0, Band ba = dense_band(),
                Band bb = dense_band(), int qlast = SQ_LAUNCHES - 1) {
    // grid: the problem's largest dimension, or the checkpoint's when the
    // host knows it (kd.dim > 0); the kernel reads each run's own dimension
    const int kmax = kd.dim > 0 ? kd.dim : p->m;
    const int Mx = M < 0 ? kmax : M, Nx = N < 0 ? kmax : N;
    GemmArgs g{A, lda, sA, B, ldb, sB, C, ldc, sC, M, N, K, kd, epi, lin, gate, sG, q, ba, bb, qlast};
    if (epi != 1 && !gate && (Mx <= 16 || Nx <= 16)) {
        int64_t gx = ((int64_t)Mx * Nx + GNT - 1) / GNT;
        if (gx > 152 * 4) gx = 152 * 4;
        k_dgemm_thin<<<dim3((unsigned)gx, (unsigned)nb), GNT, 0, p->ctx->stream>>>(g);
    } else if (waves_x_work(Mx, Nx, nb, 16) < waves_x_work(Mx, Nx, nb, GT)) {
        // 16 x 16 tiles where they spread the FP64 work more evenly over the
        // SMs (each output is summed over K in the same order: the same result)
        dim3 grd((unsigned)((Nx + 15) / 16), (unsigned)((Mx + 15) / 16), (unsigned)nb);
        k_dgemm<16><<<grd, GNT, 0, p->ctx->stream>>>(g);
    } else {
        dim3 grd((unsigned)((Nx + GT - 1) / GT), (unsigned)((Mx + GT - 1) / GT), (unsigned)nb);
        k_dgemm<GT><<<grd, GNT, 0, p->ctx->stream>>>(g);
    }
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

// e^{t dt H_k} e_1 for t = 0..steps for runs j0 .. j0+nb-1 at dimension dim
// (0: each run's m_used), the integrand rows into hlast, and (write_basis)
// the basis rows.
static int expm_large_batch(Prob* p, int j0, int nb, int dim, bool write_basis) {
    const int m = p->m, S = p->steps + 1;
    cudaStream_t st = p->ctx->stream;
    const KDim kd{p->d_state + j0, dim};
    const int64_t X_ = (int64_t)large_expm_scratch_doubles(m, p->steps);  // run stride of the scratch
    double* X = p->d_lx;
    double* X2 = X + (size_t)m * m;
    double* X3 = X2 + (size_t)m * m;
    double* X4 = X3 + (size_t)m * m;
    double* T0 = X4 + (size_t)m * m;
    double* T1 = T0 + (size_t)m * m;
    double* U = T1 + (size_t)m * m;
    double* cs = U + (size_t)m * S;
    const double* gate = cs + m;
    const double* scale = cs + m + 1;
    const int64_t sH = (int64_t)(m + 1) * m;
    const unsigned eb = (unsigned)std::min<int64_t>(((int64_t)m * m + GNT - 1) / GNT, 152 * 8);
    const dim3 ge(eb, 1, (unsigned)nb);
    k_lx_load<<<ge, GNT, 0, st>>>(p->d_H + (int64_t)j0 * sH, m, sH, X, m, X_, p->dt, kd);
    k_lx_colsum<<<dim3((unsigned)((m + 7) / 8), 1, (unsigned)nb), GNT, 0, st>>>(X, m, X_, cs, X_, kd);
    // band of H: tridiagonal when every run of the batch is a Lanczos run
    bool lanczos = true;
    for (int j = j0; j < j0 + nb; ++j) lanczos = lanczos && p->method[j] == KV_LANCZOS;
    // squaring launches: the Lanczos H has ||H_k||_1 <= 3 ||A||_2 (its alpha
    // are Rayleigh quotients and its beta norms of A v for unit v), and the
    // Taylor test passes for ||X||_1 <= 1, so with a bound of ||A||_2 at most
    // ceil(log2(3 dt bound)) squarings are needed (one more for rounding);
    // otherwise SQ_LAUNCHES.  The count is even (the result ends in `cur`).
    int L = SQ_LAUNCHES;
    if (lanczos && std::isfinite(p->sys->norm2_bound)) {
        const double nrm = 3.0 * p->dt * p->sys->norm2_bound * (1.0 + 1e-9);
        const int e = nrm > 1.0 ? (int)std::ceil(std::log2(nrm)) : 0;
        L = std::min(SQ_LAUNCHES, std::max(2, e + 1));
        L += L & 1;
    }
    k_lx_scaling<<<dim3(1, 1, (unsigned)nb), GNT, 0, st>>>(cs, X_, m, L, kd);
    k_lx_scale<<<ge, GNT, 0, st>>>(X, m, X_, scale, X_, kd);
    KV_CHECK_CUDA(cudaGetLastError());
    const Band b1 = lanczos ? Band{1, 1} : Band{1, BAND_DENSE};
    const Band b2 = band_sum(b1, b1), b3 = band_sum(b2, b1), b4 = band_sum(b2, b2);
    int rc = gemm(p, nb, X, m, X_, X, m, X_, X2, m, X_, -1, -1, -1, kd, 0, Lin4{}, nullptr, 0, 0, b1, b1);
    if (!rc) rc = gemm(p, nb, X2, m, X_, X, m, X_, X3, m, X_, -1, -1, -1, kd, 0, Lin4{}, nullptr, 0, 0, b2, b1);
    if (!rc) rc = gemm(p, nb, X2, m, X_, X2, m, X_, X4, m, X_, -1, -1, -1, kd, 0, Lin4{}, nullptr, 0, 0, b2, b2);
    if (rc) return rc;
    // Paterson-Stockmeyer: blocks B_i = c_{4i} I + c_{4i+1} X + c_{4i+2} X^2 + c_{4i+3} X^3
    double c[19];
    c[0] = 1.0;
    for (int i = 1; i <= 18; ++i) c[i] = c[i - 1] / (double)i;
    auto blk = [&](int i) {
        return Lin4{c[4 * i], c[4 * i + 1], c[4 * i + 2], 4 * i + 3 <= 18 ? c[4 * i + 3] : 0.0, X, X2,
                    4 * i + 3 <= 18 ? X3 : nullptr, m, X_};
    };
    k_lincomb<<<ge, GNT, 0, st>>>(T0, m, X_, blk(4), kd);  // B_4 = c16 I + c17 X + c18 X^2
    KV_CHECK_CUDA(cudaGetLastError());
    double* cur = T0;
    double* nxt = T1;
    Band bt = b2;  // band of B_4
    for (int i = 3; i >= 0; --i) {  // T = T X^4 + B_i
        rc = gemm(p, nb, cur, m, X_, X4, m, X_, nxt, m, X_, -1, -1, -1, kd, 1, blk(i), nullptr, 0, 0, bt, b4);
        if (rc) return rc;
        bt = band_max(band_sum(bt, b4), b3);
        std::swap(cur, nxt);
    }
    // squarings (L is even: the result ends in `cur`); launch q squares
    // only when q < s, so its operand has been squared q times
    for (int q = 0; q < L; ++q) {
        rc = gemm(p, nb, cur, m, X_, cur, m, X_, nxt, m, X_, -1, -1, -1, kd, 0, Lin4{}, gate, X_, q, bt, bt, L - 1);
        if (rc) return rc;
        bt = band_sum(bt, bt);
        std::swap(cur, nxt);
    }
    // doubling over the output steps: P_0 = E (in cur), spare buffers X2 / X3
    k_lx_init_u<<<dim3((unsigned)((m + GNT - 1) / GNT), 1, (unsigned)nb), GNT, 0, st>>>(U, S, X_, kd);
    KV_CHECK_CUDA(cudaGetLastError());
    const double* P = cur;
    double* spare[2] = {X2, X3};
    int sp = 0;
    for (int off = 1; off < S; off *= 2) {
        const int len = std::min(off, S - off);
        rc = gemm(p, nb, P, m, X_, U, S, X_, U + off, S, X_, -1, len, -1, kd);
        if (rc) return rc;
        if (2 * off < S) {
            rc = gemm(p, nb, P, m, X_, P, m, X_, spare[sp], m, X_, -1, -1, -1, kd);
            if (rc) return rc;
            P = spare[sp];
            sp ^= 1;
        }
    }
    k_lx_hlast<<<dim3((unsigned)((S + GNT - 1) / GNT), 1, (unsigned)nb), GNT, 0, st>>>(
        U, S, X_, S, p->d_hlast + (int64_t)j0 * S, kd);
    KV_CHECK_CUDA(cudaGetLastError());
    if (write_basis) {
        rc = gemm(p, nb, p->d_P + (int64_t)j0 * p->o * m, m, (int64_t)p->o * m, U, S, X_,
                  p->d_basis + (int64_t)j0 * p->o * S, S, (int64_t)p->o * S, p->o, S, -1, kd, 2);
        if (rc) return rc;
    }
    return KV_OK;
}

int launch_expm_large(Prob* p, int j0, int ncols, int dim, bool write_basis) {
    const char* name = dim > 0 ? "error_expm" : (p->expm_mode == KV_EXPM_PROPAGATE ? "expm_propagate" : "expm_large");
    LaunchScope ls(p->ctx, name);
    const int B = large_expm_batch(p->m, p->steps, p->i);
    for (int j = j0; j < j0 + ncols; j += B) {
        const int rc = expm_large_batch(p, j, std::min(B, j0 + ncols - j), dim, write_basis);
        if (rc) return rc;
    }
    return KV_OK;
}

}  // namespace kv
