/*
 * kv_oracle.c -- plain, slow, obviously-correct CPU oracle for the projected
 * Krylov verification path of "Numerical Verification of Affine Systems with up
 * to a Billion Dimensions" (Bak, Tran, Johnson).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * Everything is IEEE double precision (the paper sizes every buffer with
 * sizeof(double), Sec. 4.3), written in the order the paper states the steps:
 *
 *   ora_apply         y = A x, A a grid Laplacian (Dirichlet-0, or a coefficient
 *                     per face of the grid box) or a CSR matrix,
 *                     optionally augmented with the forcing column b and a zero
 *                     row (Sec. 2.1, affine-to-linear transformation).
 *   ora_lanczos       Lanczos with the output projection P = C V computed inside
 *                     the loop and only three n-vectors kept (Alg. 3 / Alg. 4).
 *   ora_arnoldi       Arnoldi with modified Gram-Schmidt against all previous
 *                     basis vectors (Alg. 1; the inner loop runs over the
 *                     previous vectors only), P = C V accumulated as it goes.
 *   ora_expm          matrix exponential by Pade-13 with scaling and squaring
 *                     (the library method named in Sec. 4.1; coefficients and
 *                     the scaling threshold from Higham, SIAM J. Matrix Anal.
 *                     Appl. 26(4), 2005).
 *   ora_basis         one row block of the basis matrix C e^{At} E_j per step,
 *                     ||E_j|| * P * e^{H t_k} e_1 (Eq. "approx-formula", Sec. 4.2).
 *   ora_lemma1        the a-posteriori error bound of Lemma 1 (Sec. 4.2) for a
 *                     Krylov dimension k, which Alg. 2 / Alg. 4 compare with the
 *                     error target at the dimensions 4, ceil(1.1 k), ...
 *   ora_bounds        per-step output interval over the box initial set, first
 *                     step whose upper bound reaches the unsafe half-space and the
 *                     counter-example vertex (the LP of Sec. 2.1 solved in closed
 *                     form for a box in z and one half-space per output row).
 *
 * Breakdown: the paper stops early when the new basis vector's norm is zero
 * (Sec. 4.2).  In floating point "zero" is read as ||w|| <= 1e-12 * ||A v||,
 * with ||A v|| the norm of the product before orthogonalisation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_BREAKDOWN_REL 1e-12

typedef struct {
    int kind;             /* 0: grid Laplacian, 1: CSR */
    int ndim;             /* grid: 2 or 3 */
    int64_t dims[3];      /* grid: nx, ny, nz (x fastest) */
    double coef;          /* grid: diffusion coefficient */
    double h[3];          /* grid: spacing per axis */
    int64_t n;            /* number of state variables (without augmentation) */
    const int64_t *rp;    /* CSR row pointers, n+1 */
    const int32_t *col;   /* CSR column indices */
    const double *val;    /* CSR values */
    const double *b;      /* forcing term, n entries, or NULL */
    int aug;              /* 1: the state carries the constant variable at index n */
    int trans;            /* 1: apply the transpose (A^T, or A'^T when aug) */
    const double *face;   /* grid: gamma per face (x lo, x hi, y lo, y hi, z lo, z hi),
                             2*ndim entries, or NULL for Dirichlet-0 */
} ora_op;

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops from now on (the benchmark's single-thread
 * figure); 0 or less leaves the count unchanged. */
void ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int64_t ora_dim(const ora_op *op) { return op->n + (op->aug ? 1 : 0); }

/* ---------------------------------------------------------------- A x ---- */
/* Second-order central differences: (A x)_p = coef * sum_axes
 * (x_{p-e} + x_{p+e} - 2 x_p) / h_axis^2, neighbours outside the grid are 0
 * (Dirichlet-0 boundary; semi-finite-difference model of Sec. 5.3). */
/* The grid operator with a coefficient per face of the box (the heat models
 * of Sec. 5.3 with insulated or heat-exchanging faces), term by term:
 * (A x)_p = sum over the neighbours q inside the grid of coef/h_a^2 (x_q - x_p),
 * minus gamma_f x_p for every face f the point p lies on. */
static void grid_apply_faces(const ora_op *op, const double *x, double *y) {
    const int64_t n3[3] = {op->dims[0], op->ndim >= 2 ? op->dims[1] : 1, op->ndim >= 3 ? op->dims[2] : 1};
    const int64_t stride[3] = {1, n3[0], n3[0] * n3[1]};
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < n3[2]; z++) {
        for (int64_t yy = 0; yy < n3[1]; yy++) {
            for (int64_t xx = 0; xx < n3[0]; xx++) {
                const int64_t coord[3] = {xx, yy, z};
                const int64_t p = z * stride[2] + yy * stride[1] + xx;
                const double c = x[p];
                double acc = 0.0;
                for (int a = 0; a < op->ndim; a++) {
                    const double w = op->coef / (op->h[a] * op->h[a]);
                    if (coord[a] > 0) acc += w * (x[p - stride[a]] - c);
                    else acc -= op->face[2 * a] * c;
                    if (coord[a] < n3[a] - 1) acc += w * (x[p + stride[a]] - c);
                    else acc -= op->face[2 * a + 1] * c;
                }
                y[p] = acc;
            }
        }
    }
}

static void grid_apply(const ora_op *op, const double *x, double *y) {
    if (op->face) {
        grid_apply_faces(op, x, y);
        return;
    }
    const int64_t nx = op->dims[0];
    const int64_t ny = op->ndim >= 2 ? op->dims[1] : 1;
    const int64_t nz = op->ndim >= 3 ? op->dims[2] : 1;
    double w[3] = {0, 0, 0};
    for (int a = 0; a < op->ndim; a++) w[a] = op->coef / (op->h[a] * op->h[a]);
    const int64_t sy = nx, sz = nx * ny;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < nz; z++) {
        for (int64_t yy = 0; yy < ny; yy++) {
            for (int64_t xx = 0; xx < nx; xx++) {
                const int64_t p = z * sz + yy * sy + xx;
                const double c = x[p];
                double acc = 0.0;
                {
                    double l = xx > 0 ? x[p - 1] : 0.0;
                    double r = xx < nx - 1 ? x[p + 1] : 0.0;
                    acc += w[0] * (l + r - 2.0 * c);
                }
                if (op->ndim >= 2) {
                    double l = yy > 0 ? x[p - sy] : 0.0;
                    double r = yy < ny - 1 ? x[p + sy] : 0.0;
                    acc += w[1] * (l + r - 2.0 * c);
                }
                if (op->ndim >= 3) {
                    double l = z > 0 ? x[p - sz] : 0.0;
                    double r = z < nz - 1 ? x[p + sz] : 0.0;
                    acc += w[2] * (l + r - 2.0 * c);
                }
                y[p] = acc;
            }
        }
    }
}

static void csr_apply(const ora_op *op, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < op->n; r++) {
        double acc = 0.0;
        for (int64_t e = op->rp[r]; e < op->rp[r + 1]; e++) acc += op->val[e] * x[op->col[e]];
        y[r] = acc;
    }
}

/* y = A^T x: every stored a_rc adds a_rc x_r to y_c (serial scatter). */
static void csr_apply_transpose(const ora_op *op, const double *x, double *y) {
    for (int64_t c = 0; c < op->n; c++) y[c] = 0.0;
    for (int64_t r = 0; r < op->n; r++)
        for (int64_t e = op->rp[r]; e < op->rp[r + 1]; e++) y[op->col[e]] += op->val[e] * x[r];
}

/* y = A' x with A' = [[A, b], [0, 0]] when aug (Sec. 2.1), else y = A x.
 * trans: y = A'^T x = (A^T x_{0:n}, b . x_{0:n}), the transpose dynamics of
 * Sec. 4.1 (the grid Laplacian is symmetric, A^T = A). */
void ora_apply(const ora_op *op, const double *x, double *y) {
    if (op->trans) {
        if (op->kind == 0) grid_apply(op, x, y);
        else csr_apply_transpose(op, x, y);
        if (op->aug) {
            double s = 0.0;
            if (op->b)
                for (int64_t r = 0; r < op->n; r++) s += op->b[r] * x[r];
            y[op->n] = s;
        }
        return;
    }
    if (op->kind == 0) grid_apply(op, x, y);
    else csr_apply(op, x, y);
    if (op->aug) {
        const double xa = x[op->n];
        if (op->b) {
#pragma omp parallel for schedule(static)
            for (int64_t r = 0; r < op->n; r++) y[r] += op->b[r] * xa;
        }
        y[op->n] = 0.0;
    }
}

/* ------------------------------------------------------- vector basics --- */
static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static void axpy(int64_t n, double alpha, const double *x, double *y) { /* y += alpha x */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) y[i] += alpha * x[i];
}

static void scale_into(int64_t n, double s, const double *x, double *y) { /* y = s x */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) y[i] = s * x[i];
}

/* P[:, j] = C v for the o x n output matrix C in CSR form (Sec. 3.1). */
static void project(int o, const int64_t *crp, const int64_t *ccol, const double *cval,
                    const double *v, double *P, int ldp, int j) {
    for (int r = 0; r < o; r++) {
        double s = 0.0;
        for (int64_t e = crp[r]; e < crp[r + 1]; e++) s += cval[e] * v[ccol[e]];
        P[(int64_t)r * ldp + j] = s;
    }
}

/* ------------------------------------------------------------ Lanczos ---- */
/* Alg. 3 (the three-term recurrence) with the Alg. 4 changes: the projection
 * P_{*,i} = C V_{*,i} is taken inside the loop and V_{*,i-2} is dropped, so
 * only three n-vectors are live.  Input v1 is normalised.  Output H is dense
 * (m+1) x m row-major: H[j][j] = alpha_j, H[j+1][j] = H[j][j+1] = beta_{j+1};
 * H[m][m-1] is the discarded extra row (kept for diagnostics).  P is o x m.
 * Returns the number of columns of H / P that are valid (m, or fewer after a
 * breakdown, when the Krylov space is invariant and the result is exact). */
int ora_lanczos(const ora_op *op, const double *v1, int m, int o, const int64_t *crp,
                const int64_t *ccol, const double *cval, double *H, double *P) {
    const int64_t N = ora_dim(op);
    double *vprev = (double *)calloc((size_t)N, sizeof(double));
    double *v = (double *)malloc((size_t)N * sizeof(double));
    double *w = (double *)malloc((size_t)N * sizeof(double));
    memset(H, 0, sizeof(double) * (size_t)(m + 1) * m);
    memcpy(v, v1, sizeof(double) * (size_t)N);
    project(o, crp, ccol, cval, v, P, m, 0);
    int used = m;
    for (int j = 0; j < m; j++) {
        ora_apply(op, v, w);                                   /* w = A v_j            */
        const double nAv = sqrt(dot(N, w, w));
        if (j > 0) {
            H[(int64_t)(j - 1) * m + j] = H[(int64_t)j * m + (j - 1)];
            axpy(N, -H[(int64_t)(j - 1) * m + j], vprev, w);   /* w -= beta_j v_{j-1}  */
        }
        H[(int64_t)j * m + j] = dot(N, v, w);                  /* alpha_j = v_j . w    */
        axpy(N, -H[(int64_t)j * m + j], v, w);                 /* w -= alpha_j v_j     */
        const double beta = sqrt(dot(N, w, w));                /* beta_{j+1} = ||w||   */
        H[(int64_t)(j + 1) * m + j] = beta;
        if (beta <= ORA_BREAKDOWN_REL * nAv) { used = j + 1; break; }
        double *t = vprev; vprev = v; v = t;                   /* drop v_{j-1}          */
        scale_into(N, 1.0 / beta, w, v);                       /* v_{j+1} = w / beta    */
        if (j + 1 < m) project(o, crp, ccol, cval, v, P, m, j + 1);
    }
    free(vprev); free(v); free(w);
    return used;
}

/* ------------------------------------------------------------ Arnoldi ---- */
/* Alg. 1: V_{*,i} = A V_{*,i-1}, then for every previous basis vector j:
 * H_{j,i-1} = V_j . V_i and V_i -= H_{j,i-1} V_j (modified Gram-Schmidt),
 * H_{i,i-1} = ||V_i||, V_i /= H_{i,i-1}.  The basis (m+1 vectors) is stored,
 * as Arnoldi must (Eq. memory_arnoldi).  H is (m+1) x m row-major, P is o x m.
 * Returns the number of valid columns. */
int ora_arnoldi(const ora_op *op, const double *v1, int m, int o, const int64_t *crp,
                const int64_t *ccol, const double *cval, double *H, double *P) {
    const int64_t N = ora_dim(op);
    double *V = (double *)malloc((size_t)N * (size_t)(m + 1) * sizeof(double));
    double *w = (double *)malloc((size_t)N * sizeof(double));
    memset(H, 0, sizeof(double) * (size_t)(m + 1) * m);
    memcpy(V, v1, sizeof(double) * (size_t)N);
    project(o, crp, ccol, cval, V, P, m, 0);
    int used = m;
    for (int j = 0; j < m; j++) {
        ora_apply(op, V + (int64_t)j * N, w);
        const double nAv = sqrt(dot(N, w, w));
        for (int l = 0; l <= j; l++) {
            const double hl = dot(N, V + (int64_t)l * N, w);
            H[(int64_t)l * m + j] = hl;
            axpy(N, -hl, V + (int64_t)l * N, w);
        }
        const double beta = sqrt(dot(N, w, w));
        H[(int64_t)(j + 1) * m + j] = beta;
        if (beta <= ORA_BREAKDOWN_REL * nAv) { used = j + 1; break; }
        scale_into(N, 1.0 / beta, w, V + (int64_t)(j + 1) * N);
        if (j + 1 < m) project(o, crp, ccol, cval, V + (int64_t)(j + 1) * N, P, m, j + 1);
    }
    free(V); free(w);
    return used;
}

/* --------------------------------------------------------------- expm ---- */
static void matmul(int m, const double *A, const double *B, double *C) {
    for (int i = 0; i < m; i++) {
        for (int j = 0; j < m; j++) C[i * m + j] = 0.0;
        for (int k = 0; k < m; k++) {
            const double a = A[i * m + k];
            for (int j = 0; j < m; j++) C[i * m + j] += a * B[k * m + j];
        }
    }
}

/* Solve Q X = R (m x m, m right-hand sides) by Gaussian elimination with
 * partial pivoting; Q and R are overwritten, the solution is left in R. */
static void solve_inplace(int m, double *Q, double *R) {
    for (int k = 0; k < m; k++) {
        int p = k;
        double best = fabs(Q[k * m + k]);
        for (int i = k + 1; i < m; i++)
            if (fabs(Q[i * m + k]) > best) { best = fabs(Q[i * m + k]); p = i; }
        if (p != k) {
            for (int j = 0; j < m; j++) {
                double t = Q[k * m + j]; Q[k * m + j] = Q[p * m + j]; Q[p * m + j] = t;
                t = R[k * m + j]; R[k * m + j] = R[p * m + j]; R[p * m + j] = t;
            }
        }
        for (int i = k + 1; i < m; i++) {
            const double f = Q[i * m + k] / Q[k * m + k];
            if (f == 0.0) continue;
            for (int j = k; j < m; j++) Q[i * m + j] -= f * Q[k * m + j];
            for (int j = 0; j < m; j++) R[i * m + j] -= f * R[k * m + j];
        }
    }
    for (int k = m - 1; k >= 0; k--) {
        for (int j = 0; j < m; j++) {
            double s = R[k * m + j];
            for (int i = k + 1; i < m; i++) s -= Q[k * m + i] * R[i * m + j];
            R[k * m + j] = s / Q[k * m + k];
        }
    }
}

/* Pade coefficients of degree 13 normalised so that b_13 = 1:
 * b_j = (26 - j)! / (j! (13 - j)!), an integer (Higham 2005). */
static void pade13_coeffs(double b[14]) {
    for (int j = 0; j <= 13; j++) {
        /* (26-j)!/(13-j)! is the product of the 13 integers 14-j .. 26-j */
        unsigned long long num = 1ULL;
        for (int k = 14 - j; k <= 26 - j; k++) num *= (unsigned long long)k;
        unsigned long long den = 1ULL;
        for (int k = 2; k <= j; k++) den *= (unsigned long long)k;
        b[j] = (double)(num / den);
    }
}

/* E = exp(A) for an m x m row-major A: scale A by 2^-s so that its 1-norm is
 * at most theta_13 = 5.371920351148152 (Higham 2005, Table 2.3), evaluate the
 * [13/13] Pade approximant r(X) = q(X)^{-1} p(X), then square s times. */
void ora_expm(int m, const double *A, double *E) {
    const double theta13 = 5.371920351148152;
    double b[14];
    pade13_coeffs(b);
    const size_t mm = (size_t)m * m;
    double *X = (double *)malloc(mm * sizeof(double));
    double *X2 = (double *)malloc(mm * sizeof(double));
    double *X4 = (double *)malloc(mm * sizeof(double));
    double *X6 = (double *)malloc(mm * sizeof(double));
    double *T = (double *)malloc(mm * sizeof(double));
    double *U = (double *)malloc(mm * sizeof(double));
    double *V = (double *)malloc(mm * sizeof(double));

    double norm1 = 0.0;
    for (int j = 0; j < m; j++) {
        double s = 0.0;
        for (int i = 0; i < m; i++) s += fabs(A[i * m + j]);
        if (s > norm1) norm1 = s;
    }
    int s = 0;
    if (norm1 > theta13) s = (int)ceil(log2(norm1 / theta13));
    const double sc = ldexp(1.0, -s);
    for (size_t k = 0; k < mm; k++) X[k] = A[k] * sc;
    matmul(m, X, X, X2);
    matmul(m, X2, X2, X4);
    matmul(m, X4, X2, X6);
    /* U = X [ X6 (b13 X6 + b11 X4 + b9 X2) + b7 X6 + b5 X4 + b3 X2 + b1 I ] */
    for (size_t k = 0; k < mm; k++) T[k] = b[13] * X6[k] + b[11] * X4[k] + b[9] * X2[k];
    matmul(m, X6, T, U);
    for (size_t k = 0; k < mm; k++) U[k] += b[7] * X6[k] + b[5] * X4[k] + b[3] * X2[k];
    for (int i = 0; i < m; i++) U[i * m + i] += b[1];
    memcpy(T, U, mm * sizeof(double));
    matmul(m, X, T, U);
    /* V = X6 (b12 X6 + b10 X4 + b8 X2) + b6 X6 + b4 X4 + b2 X2 + b0 I */
    for (size_t k = 0; k < mm; k++) T[k] = b[12] * X6[k] + b[10] * X4[k] + b[8] * X2[k];
    matmul(m, X6, T, V);
    for (size_t k = 0; k < mm; k++) V[k] += b[6] * X6[k] + b[4] * X4[k] + b[2] * X2[k];
    for (int i = 0; i < m; i++) V[i * m + i] += b[0];
    /* (V - U) R = (V + U) */
    for (size_t k = 0; k < mm; k++) { T[k] = V[k] - U[k]; E[k] = V[k] + U[k]; }
    solve_inplace(m, T, E);
    for (int q = 0; q < s; q++) {
        matmul(m, E, E, T);
        memcpy(E, T, mm * sizeof(double));
    }
    free(X); free(X2); free(X4); free(X6); free(T); free(U); free(V);
}

/* -------------------------------------------------------------- basis ---- */
/* For one column with Krylov data (H, P, mu valid columns) and beta0 = ||E_j||:
 * out[r][k] = beta0 * sum_l P[r][l] (e^{H_mu t_k})[l][0],  t_k = k dt,
 * k = 0..steps (Eq. approx-formula: e^{At} v ~ ||v|| V_k e^{H_k t} e_1, then
 * projected by C).  H is (ldh+1) x ldh row-major, P is o x ldh. */
void ora_basis(int mu, int ldh, const double *H, int o, const double *P, double beta0,
               double dt, int steps, double *out) {
#pragma omp parallel
    {
        double *X = (double *)malloc(sizeof(double) * (size_t)mu * mu);
        double *E = (double *)malloc(sizeof(double) * (size_t)mu * mu);
#pragma omp for schedule(dynamic, 4)
        for (int k = 0; k <= steps; k++) {
            const double t = (double)k * dt;
            for (int i = 0; i < mu; i++)
                for (int j = 0; j < mu; j++) X[i * mu + j] = H[(int64_t)i * ldh + j] * t;
            ora_expm(mu, X, E);
            for (int r = 0; r < o; r++) {
                double s = 0.0;
                for (int l = 0; l < mu; l++) s += P[(int64_t)r * ldh + l] * E[l * mu + 0];
                out[(int64_t)r * (steps + 1) + k] = beta0 * s;
            }
        }
        free(X); free(E);
    }
}

/* -------------------------------------------------------- error bound ---- */
/* Lemma 1 (Sec. 4.2, after Wang and Ye) for the Krylov pair (V_k, H_k) of a
 * unit start vector v, applied with B = -A as the paper prescribes:
 *   || e^{tA} v - V_k e^{t H_k} e_1 || <= h_{k+1,k} e^{max(mu,0) T} int_0^T |h(t)| dt
 * with h(t) = e_k^T e^{t H_k} e_1, T = steps * dt, and mu an upper bound of the
 * largest eigenvalue of (A + A^T)/2 (the lemma's nu is the smallest eigenvalue
 * of (B + B^T)/2 = -(A + A^T)/2, so -min(nu, 0) = max(mu, 0)).  Arnoldi on -A
 * gives H_k(-A) = -D H_k(A) D, D = diag(1, -1, 1, ...), so |h| is the same for
 * both matrices.  The integral is the composite trapezoid rule on the output
 * grid t_j = j dt, j = 0..steps, with e^{t_j H_k} e_1 from the Pade exponential
 * of t_j H_k.  H is row-major with leading dimension ldh (k <= ldh); hk1 is
 * h_{k+1,k}.  Returns the bound (0 when hk1 = 0: the space is invariant). */
double ora_lemma1(int k, int ldh, const double *H, double hk1, double mu, double dt, int steps) {
    if (k <= 0 || hk1 == 0.0) return 0.0;
    double *hv = (double *)malloc(sizeof(double) * (size_t)(steps + 1));
#pragma omp parallel
    {
        double *X = (double *)malloc(sizeof(double) * (size_t)k * k);
        double *E = (double *)malloc(sizeof(double) * (size_t)k * k);
#pragma omp for schedule(dynamic, 4)
        for (int j = 0; j <= steps; j++) {
            const double t = (double)j * dt;
            for (int r = 0; r < k; r++)
                for (int c = 0; c < k; c++) X[r * k + c] = H[(int64_t)r * ldh + c] * t;
            ora_expm(k, X, E);
            hv[j] = fabs(E[(k - 1) * k + 0]);   /* row k, column 1 */
        }
        free(X); free(E);
    }
    double integral = 0.0;
    for (int j = 1; j <= steps; j++) integral += 0.5 * dt * (hv[j - 1] + hv[j]);
    free(hv);
    const double T = (double)steps * dt;
    return hk1 * exp((mu > 0.0 ? mu : 0.0) * T) * integral;
}

/* ------------------------------------------------------------- bounds ---- */
/* basis is ncol x o x (steps+1): the basis matrix C e^{A t_k} E per step.
 * With z_j in [zlo_j, zhi_j], y_r(t_k) = sum_j basis[j][r][k] z_j ranges over
 * [sum_j min(p zlo_j, p zhi_j), sum_j max(p zlo_j, p zhi_j)] -- the optimum of
 * the per-step LP of Sec. 2.1 for a box initial set and a half-space
 * y_r >= theta_r.  The first violation is the smallest step k, then the
 * smallest row r, with hi_r(k) >= theta_r (t = k dt <= T, k = 0 included).
 * The counter-example is the maximising vertex: z_j = zhi_j if p > 0, zlo_j if
 * p < 0, the midpoint if p == 0; ystar = hi_r(k).  Returns 1 if unsafe. */
int ora_bounds(int o, int ncol, int steps, const double *basis, const double *zlo,
               const double *zhi, const double *theta, double *lo, double *hi,
               int *viol_step, int *viol_row, double *zstar, double *ystar) {
    const int64_t S = steps + 1;
    *viol_step = -1;
    *viol_row = -1;
    for (int k = 0; k <= steps; k++) {
        for (int r = 0; r < o; r++) {
            double l = 0.0, h = 0.0;
            for (int j = 0; j < ncol; j++) {
                const double p = basis[((int64_t)j * o + r) * S + k];
                const double a = p * zlo[j], c = p * zhi[j];
                l += a < c ? a : c;
                h += a < c ? c : a;
            }
            lo[(int64_t)r * S + k] = l;
            hi[(int64_t)r * S + k] = h;
            if (*viol_step < 0 && h >= theta[r]) { *viol_step = k; *viol_row = r; }
        }
    }
    if (*viol_step < 0) return 0;
    const int k = *viol_step, r = *viol_row;
    for (int j = 0; j < ncol; j++) {
        const double p = basis[((int64_t)j * o + r) * S + k];
        zstar[j] = p > 0 ? zhi[j] : (p < 0 ? zlo[j] : 0.5 * (zlo[j] + zhi[j]));
    }
    *ystar = hi[(int64_t)r * S + k];
    return 1;
}
