// k_expm.cu -- batched FP64 exponential of the small Krylov matrix H and the
// basis-matrix rows C e^{A t_k} E_j ~ ||E_j|| P e^{H t_k} e_1 (Eq.
// approx-formula, Sec. 4.2).
//
// The exponential is the [13/13] Pade approximant with scaling and squaring
// (the off-the-shelf method named in Sec. 4.1; degree-13 coefficients
// b_j = (26-j)! / (j! (13-j)!) and the threshold theta_13 = 5.371920351148152
// from Higham, SIAM J. Matrix Anal. Appl. 26(4), 2005).  One CTA owns one
// matrix in shared memory; all arithmetic is double.
//
// Two schedules (kv_problem_desc.expm_mode):
//   PER_STEP   one CTA per (column, step): e^{H t_k} for every k (this file,
//              dimensions up to 64).
//   PROPAGATE  M = e^{H dt}, u_k = M^k e_1: the same vectors in exact
//              arithmetic, by GEMM doubling over the steps (k_expm_large.cu,
//              which also takes every dimension above 64).
//
// Both also record |(u_k)_mu|, the last entry of u_k = e^{t_k H_mu} e_1: the
// integrand of the a-posteriori bound of Lemma 1 (Sec. 4.2), which
// k_error_bound integrates by the trapezoid rule over the output grid.  For
// the error control of Alg. 2 / Alg. 4 the same kernels run on the leading
// k x k block of H at the checkpoint dimensions (dim = k, no basis output).
#include <math.h>

#include "kv_internal.h"

namespace kv {

constexpr int ENT = 256;

__constant__ double c_pade13[14];

// C = A B for n x n row-major matrices in shared memory (ld = n); C must not
// alias A or B.  Ends with a barrier.
__device__ void smm(int n, const double* A, const double* B, double* C) {
    const int nn = n * n;
    for (int e = threadIdx.x; e < nn; e += ENT) {
        const int i = e / n, j = e - i * n;
        double s = 0.0;
        const double* a = A + i * n;
        for (int k = 0; k < n; ++k) s = fma(a[k], B[k * n + j], s);
        C[e] = s;
    }
    __syncthreads();
}

// Solve Q X = R in place (X left in R), Gaussian elimination with partial
// pivoting.  piv / fac are shared scratch of n entries.  Ends with a barrier.
__device__ void ssolve(int n, double* Q, double* R, double* fac, int* piv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < n; ++k) {
        if (warp == 0) {
            double best = -1.0;
            int bi = k;
            for (int i = k + lane; i < n; i += 32) {
                const double a = fabs(Q[i * n + k]);
                if (a > best) { best = a; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) *piv = bi;
        }
        __syncthreads();
        const int p = *piv;
        if (p != k) {
            for (int c = threadIdx.x; c < 2 * n; c += ENT) {
                double* M = c < n ? Q : R;
                const int cc = c < n ? c : c - n;
                const double t = M[k * n + cc];
                M[k * n + cc] = M[p * n + cc];
                M[p * n + cc] = t;
            }
            __syncthreads();
        }
        const double dk = Q[k * n + k];
        for (int i = k + 1 + threadIdx.x; i < n; i += ENT) fac[i] = Q[i * n + k] / dk;
        __syncthreads();
        const int rows = n - k - 1;
        const int cols = 2 * n;  // Q columns k+1..n-1 and all of R (waste on Q's left part is skipped)
        for (int e = threadIdx.x; e < rows * cols; e += ENT) {
            const int i = k + 1 + e / cols, c = e % cols;
            const double f = fac[i];
            if (c < n) {
                if (c > k) Q[i * n + c] = fma(-f, Q[k * n + c], Q[i * n + c]);
            } else {
                const int cc = c - n;
                R[i * n + cc] = fma(-f, R[k * n + cc], R[i * n + cc]);
            }
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        for (int c = threadIdx.x; c < n; c += ENT) {
            double s = R[k * n + c];
            for (int i = k + 1; i < n; ++i) s = fma(-Q[k * n + i], R[i * n + c], s);
            R[k * n + c] = s / Q[k * n + k];
        }
        __syncthreads();
    }
}

// exp(X) for the n x n matrix in buf[0]; six n x n buffers buf[0..5].
// Returns the index of the buffer holding the result.
__device__ int sexpm(int n, double* buf[6], double* fac, int* piv, double* red) {
    double *X = buf[0], *X2 = buf[1], *X4 = buf[2], *X6 = buf[3], *T = buf[4], *U = buf[5];
    const double* b = c_pade13;
    // 1-norm (max column abs sum)
    double cmax = 0.0;
    for (int j = threadIdx.x; j < n; j += ENT) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(X[i * n + j]);
        cmax = fmax(cmax, s);
    }
    for (int o = 16; o > 0; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cmax;
    __syncthreads();
    double norm1 = 0.0;
    for (int w = 0; w < ENT / 32; ++w) norm1 = fmax(norm1, red[w]);
    const double theta13 = 5.371920351148152;
    // squarings; a non-finite or absurd norm (> theta13 * 2^200) gets no
    // scaling so the result is NaN/inf instead of an unbounded loop
    int s = 0;
    if (norm1 > theta13 && norm1 < theta13 * 1.6e60) s = (int)ceil(log2(norm1 / theta13));
    if (s > 0) {
        const double sc = ldexp(1.0, -s);
        for (int e = threadIdx.x; e < n * n; e += ENT) X[e] *= sc;
    }
    __syncthreads();
    smm(n, X, X, X2);
    smm(n, X2, X2, X4);
    smm(n, X4, X2, X6);
    for (int e = threadIdx.x; e < n * n; e += ENT) T[e] = b[13] * X6[e] + b[11] * X4[e] + b[9] * X2[e];
    __syncthreads();
    smm(n, X6, T, U);
    for (int e = threadIdx.x; e < n * n; e += ENT) {
        U[e] += b[7] * X6[e] + b[5] * X4[e] + b[3] * X2[e];
        if (e / n == e % n) U[e] += b[1];
    }
    __syncthreads();
    smm(n, X, U, T);  // T = odd part
    for (int e = threadIdx.x; e < n * n; e += ENT) U[e] = b[12] * X6[e] + b[10] * X4[e] + b[8] * X2[e];
    __syncthreads();
    smm(n, X6, U, X);  // X = X6 (...)
    for (int e = threadIdx.x; e < n * n; e += ENT) {
        X[e] += b[6] * X6[e] + b[4] * X4[e] + b[2] * X2[e];
        if (e / n == e % n) X[e] += b[0];
    }
    __syncthreads();
    // Q = V - U into X2, R = V + U into X4
    for (int e = threadIdx.x; e < n * n; e += ENT) {
        X2[e] = X[e] - T[e];
        X4[e] = X[e] + T[e];
    }
    __syncthreads();
    ssolve(n, X2, X4, fac, piv);
    int cur = 2, spare = 3;
    for (int q = 0; q < s; ++q) {
        smm(n, buf[cur], buf[cur], buf[spare]);
        const int t = cur;
        cur = spare;
        spare = t;
    }
    return cur;
}

struct ExpmArgs {
    const double* H;       // i x (m+1) x m
    const double* P;       // i x o x m
    const ColState* st;    // i
    double* basis;         // i x o x (steps+1)
    int m, o, steps;
    double dt;
    double* hlast;         // i x (steps+1): |(e^{t_k H_mu} e_1)_mu|
    int dim;               // 0: each column's m_used, basis written; k > 0: H_k, columns not done only
    int j0;                // first column of the launch
};

// Dimension a column is evaluated at, or 0 to skip it (a checkpoint of a
// column that has stopped already).
__device__ __forceinline__ int eval_dim(const ExpmArgs& a, int j) {
    if (a.dim > 0) return a.st[j].done ? -1 : a.dim;
    return a.st[j].m_used;
}

__device__ void load_scaled_H(const ExpmArgs& a, int j, int mu, double t, double* X) {
    const double* H = a.H + (int64_t)j * (a.m + 1) * a.m;
    for (int e = threadIdx.x; e < mu * mu; e += ENT) {
        const int r = e / mu, c = e - r * mu;
        X[e] = H[(int64_t)r * a.m + c] * t;
    }
    __syncthreads();
}

// out[r] = beta0 * P[r, 0:mu] . u  (u has stride `stride`), one warp per row
__device__ void project_rows(const ExpmArgs& a, int j, int mu, const double* u, int stride, int k) {
    const double* P = a.P + (int64_t)j * a.o * a.m;
    const double b0 = a.st[j].beta0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < a.o; r += ENT / 32) {
        double s = 0.0;
        for (int l = lane; l < mu; l += 32) s = fma(P[(int64_t)r * a.m + l], u[l * stride], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) a.basis[((int64_t)j * a.o + r) * (a.steps + 1) + k] = b0 * s;
    }
}

__global__ void __launch_bounds__(ENT) k_expm_per_step(ExpmArgs a) {
    extern __shared__ double smem[];
    __shared__ double fac[EXPM_SMEM_M];
    __shared__ int piv;
    __shared__ double red[ENT / 32];
    const int j = a.j0 + blockIdx.y;
    const int mu = eval_dim(a, j);
    if (mu < 0) return;
    double* hl = a.hlast + (int64_t)j * (a.steps + 1);
    for (int k = blockIdx.x; k <= a.steps; k += gridDim.x) {
        if (mu == 0) {
            if (a.dim == 0)
                for (int r = threadIdx.x; r < a.o; r += ENT) a.basis[((int64_t)j * a.o + r) * (a.steps + 1) + k] = 0.0;
            if (threadIdx.x == 0) hl[k] = 0.0;
            continue;
        }
        double* buf[6];
        for (int q = 0; q < 6; ++q) buf[q] = smem + q * mu * mu;
        load_scaled_H(a, j, mu, (double)k * a.dt, buf[0]);
        const int res = sexpm(mu, buf, fac, &piv, red);
        if (threadIdx.x == 0) hl[k] = fabs(buf[res][(mu - 1) * mu]);  // row mu, column 1
        if (a.dim == 0) project_rows(a, j, mu, buf[res], mu, k);  // first column: stride mu
        __syncthreads();
    }
}

struct ErrArgs {
    const double* H;       // i x (m+1) x m
    ColState* st;          // i
    const double* hlast;   // i x (steps+1)
    double* err;           // i
    const int* aug;        // i, or null: column works on A' (carries the constant)
    double mu, mu_aug;     // log-norm bounds of A and A'
    int m, steps;
    double dt, eps;
    int dim, j0;
};

// Lemma 1 (Sec. 4.2) with B = -A: err = h_{k+1,k} e^{max(mu,0) T} times the
// trapezoid sum of |h(t_j)| over the output grid.  One CTA per column; the
// partial sums are combined in a fixed order.  At a checkpoint (dim = k) a
// column whose bound is below eps stops: done = 1, m_used = k (Alg. 2 /
// Alg. 4), and the Krylov launches that follow return at once.
__global__ void __launch_bounds__(ENT) k_error_bound(ErrArgs a) {
    __shared__ double red[ENT / 32];
    const int j = a.j0 + blockIdx.x;
    ColState* st = a.st + j;
    if (a.dim > 0 && st->done) return;
    const int mu = a.dim > 0 ? a.dim : st->m_used;
    const double* hl = a.hlast + (int64_t)j * (a.steps + 1);
    double s = 0.0;
    if (mu > 0)
        for (int k = 1 + threadIdx.x; k <= a.steps; k += ENT) s += 0.5 * a.dt * (hl[k - 1] + hl[k]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double integral = 0.0;
    for (int w = 0; w < ENT / 32; ++w) integral += red[w];
    double err = 0.0;
    if (mu > 0) {
        const double hk1 = a.H[((int64_t)j * (a.m + 1) + mu) * a.m + (mu - 1)];
        const double mu_col = (a.aug && a.aug[j]) ? a.mu_aug : a.mu;
        if (hk1 != 0.0) err = hk1 * exp(fmax(mu_col, 0.0) * a.steps * a.dt) * integral;
    }
    a.err[j] = err;
    if (a.dim > 0 && err < a.eps) {
        st->m_used = a.dim;
        st->done = 1;
    }
}

static bool g_coeffs_ready[64] = {false};

static int upload_coeffs(int device) {
    if (device >= 0 && device < 64 && g_coeffs_ready[device]) return KV_OK;
    double b[14];
    for (int j = 0; j <= 13; ++j) {
        // (26-j)!/(13-j)! = product of the 13 integers 14-j .. 26-j; divide by j!
        unsigned long long num = 1ULL, den = 1ULL;
        for (int k = 14 - j; k <= 26 - j; ++k) num *= (unsigned long long)k;
        for (int k = 2; k <= j; ++k) den *= (unsigned long long)k;
        b[j] = (double)(num / den);
    }
    KV_CHECK_CUDA(cudaMemcpyToSymbol(c_pade13, b, sizeof(b)));
    if (device >= 0 && device < 64) g_coeffs_ready[device] = true;
    return KV_OK;
}

// One-time set-up per process and device: the Pade coefficients in constant
// memory and the shared-memory limit of both kernels (for the largest m).
// Neither may run during stream capture, so graph capture calls this first.
int expm_prepare(int device) {
    int rc = upload_coeffs(device);
    if (rc != KV_OK) return rc;
    static bool attr_set = false;
    if (!attr_set) {
        const int smax = 6 * EXPM_SMEM_M * EXPM_SMEM_M * (int)sizeof(double);
        KV_CHECK_CUDA(cudaFuncSetAttribute(k_expm_per_step, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
        attr_set = true;
    }
    return KV_OK;
}

// The exponentials of columns j0 .. j0+ncols-1 at dimension dim (0: each
// column's m_used, with the basis rows).
static int launch_expm(Prob* p, int j0, int ncols, int dim) {
    const int mm = dim > 0 ? dim : p->m;
    if (p->expm_mode == KV_EXPM_PROPAGATE || mm > EXPM_SMEM_M) return launch_expm_large(p, j0, ncols, dim, dim == 0);
    int rc = expm_prepare(p->ctx->device);
    if (rc != KV_OK) return rc;
    ExpmArgs a{p->d_H, p->d_P, p->d_state, p->d_basis, p->m, p->o, p->steps, p->dt, p->d_hlast, dim, j0};
    const size_t smem = (size_t)6 * mm * mm * sizeof(double);
    {
        int gx = p->steps + 1;
        if (gx > 65535 * 16) gx = 65535 * 16;
        dim3 grd((unsigned)gx, (unsigned)ncols);
        LaunchScope ls(p->ctx, dim > 0 ? "error_expm" : "expm_per_step");
        k_expm_per_step<<<grd, ENT, smem, p->ctx->stream>>>(a);
    }
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

static int launch_bound(Prob* p, int j0, int ncols, int dim) {
    ErrArgs e{p->d_H, p->d_state, p->d_hlast, p->d_err, p->sys->kind == 1 ? p->d_aug : nullptr,
              p->sys->mu, p->sys->mu_aug, p->m, p->steps, p->dt, p->err_target, dim, j0};
    LaunchScope ls(p->ctx, "error_bound");
    k_error_bound<<<ncols, ENT, 0, p->ctx->stream>>>(e);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

int launch_expm_basis(Prob* p) { return launch_expm(p, 0, p->i, 0); }

int launch_error_check(Prob* p, int j0, int ncols, int dim) {
    const int rc = launch_expm(p, j0, ncols, dim);
    return rc ? rc : launch_bound(p, j0, ncols, dim);
}

int launch_error_final(Prob* p) { return launch_bound(p, 0, p->i, 0); }

}  // namespace kv
