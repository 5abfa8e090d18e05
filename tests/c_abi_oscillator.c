/* A C11 client of libkv: the timed harmonic oscillator of Sec. 2.2 through
 * the C ABI alone (no C++ and no Python between the caller and the library).
 *
 * x' = y, y' = -x, t' = 1 as x' = A x + b with b = (0, 0, 1); initial set
 * x0 = -5, y0 in [0, 1], t0 = 0 (the fixed column (-5, 0, 0) carries the
 * constant variable, the generator (0, 1, 0) has z in [0, 1]); output x,
 * unsafe x >= 4, step pi/4, four steps.  Prints one line of key=value pairs
 * and returns 0, or prints the library's error message and returns 1. */
#include <math.h>
#include <stdio.h>

#include "kv.h"

static int check(int rc, const char *what) {
    if (rc != KV_OK) {
        fprintf(stderr, "%s failed (%d): %s\n", what, rc, kv_last_error());
        return 1;
    }
    return 0;
}

int main(void) {
    const double pi = 3.14159265358979323846;
    const int64_t rp[4] = {0, 1, 2, 2};
    const int32_t col[2] = {1, 0};
    const double val[2] = {1.0, -1.0};
    const double b[3] = {0.0, 0.0, 1.0};
    const double gen[3] = {0.0, 1.0, 0.0};
    const double fix[3] = {-5.0, 0.0, 0.0};
    const int64_t crp[2] = {0, 1};
    const int64_t ccol[1] = {0};
    const double cval[1] = {1.0};
    const double theta[1] = {4.0};
    kv_column cols[2] = {{0}, {0}};
    kv_problem_desc d = {0};
    kv_ctx *ctx = NULL;
    kv_sys *sys = NULL;
    kv_prob *prob = NULL;
    double lo[5], hi[5], basis[2 * 5], beta0[2], zstar[2];
    int32_t m_used[2];
    kv_result res = {0};
    int k;

    cols[0].kind = KV_COL_DENSE;
    cols[0].zlo = 0.0;
    cols[0].zhi = 1.0;
    cols[0].dense = gen;
    cols[1].kind = KV_COL_DENSE;
    cols[1].is_fixed = 1;
    cols[1].zlo = 1.0;
    cols[1].zhi = 1.0;
    cols[1].dense = fix;
    d.i = 2;
    d.cols = cols;
    d.o = 1;
    d.c_row_ptr = crp;
    d.c_col = ccol;
    d.c_val = cval;
    d.theta = theta;
    d.dt = pi / 4.0;
    d.steps = 4;
    d.krylov_m = 4;
    d.method = KV_ARNOLDI;
    d.expm_mode = KV_EXPM_PER_STEP;
    d.simulate = KV_SIM_FORWARD;

    res.lo = lo;
    res.hi = hi;
    res.basis = basis;
    res.beta0 = beta0;
    res.m_used = m_used;
    res.z_star = zstar;

    if (check(kv_create(&ctx, 0, NULL, (size_t)64 << 20, NULL), "kv_create")) return 1;
    if (check(kv_system_csr(ctx, &sys, 3, rp, col, val, b, 0, KV_FP64, 0), "kv_system_csr")) return 1;
    if (check(kv_problem(ctx, &prob, sys, &d, KV_FP64), "kv_problem")) return 1;
    if (check(kv_run(prob, &res), "kv_run")) return 1;
    printf("violation_step=%d violation_row=%d y_star=%.6f", res.first_violation_step, res.violation_row,
           res.y_star);
    printf(" m_used_gen=%d m_used_fix=%d", m_used[0], m_used[1]);
    /* basis [j][r][k]: C e^{A t_k} E_j for the generator (j = 0) and the fixed column (j = 1) */
    for (k = 0; k <= 4; ++k) printf(" basis_gen_%d=%.9f basis_fix_%d=%.9f", k, basis[k], k, basis[5 + k]);
    printf(" z_gen=%.6f\n", zstar[0]);
    kv_prob_destroy(prob);
    kv_sys_destroy(sys);
    kv_destroy(ctx);
    return isfinite(hi[4]) ? 0 : 1;
}
