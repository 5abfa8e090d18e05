// k_lp.cu -- the per-step LP of Sec. 2.1 for polyhedral initial and unsafe
// sets, over the projected basis B_k = C e^{A t_k} E (Sec. 3.1-3.2).
//
// Step k asks for
//     t*_k = min t   over (z, t)
//            s.t.    U_u B_k z - t <= upsilon_u   (unsafe rows, unit norm)
//                    I_q z         <= iota_q      (extra initial-set rows)
//                    lo <= z <= hi                (the columns' boxes)
// the largest normalised violation of the unsafe constraints that the
// initial set can bring down to; the unsafe set is reachable at step k iff
// t*_k <= tol, and the minimiser z* is a counter-example.
//
// One CTA per step solves the dual of that LP,
//     min b^T y   s.t.   A^T y = -c,  y >= 0      (c = e_t),
// by the two-phase dense simplex method (Dantzig pricing, Harris ratio test,
// Bland's rule against cycling) on a tableau in shared memory: d = i + 1
// equality rows (one per primal variable), one column per primal constraint
// scaled to unit norm (the same half-space), d artificial columns and the
// right-hand side.  The minimiser (z*, t*) is the simplex multiplier vector,
// read from the reduced costs of the artificial columns.
//
// The tableau is kept in double-double arithmetic (each entry an unevaluated
// sum hi + lo of two doubles, about 106 bits).  Outputs that depend only
// weakly on some columns of E (a basis entry of 1e-7 next to the unit t
// coefficient) force small but genuine pivots, whose element growth turns
// exact zeros into double-precision noise of 1e-11 that a later pivot can
// take for a real entry; at 106 bits that noise is ~1e-27, far below the
// pivot threshold, while genuine entries of 1e-12 stay usable.
#include <limits.h>
#include <math.h>

#include "kv_internal.h"

namespace kv {

constexpr int LNT = 256;
constexpr double LP_EPS_PIV = 1e-13;   // smallest usable pivot (columns start with unit norm)
constexpr double LP_EPS_FEAS = 1e-9;   // phase-1 optimum above this: the dual is infeasible
// Reduced costs and right-hand sides are double-double accurate, so the
// entering threshold can resolve improvements of the margin far below the
// size of the basis entries (a generator that moves the outputs by 1e-7
// changes the margin by ~1e-10).
constexpr double LP_EPS_RC = 1e-14;    // entering threshold on reduced costs (x the largest cost in phase 2)
constexpr double LP_HARRIS = 1e-14;    // right-hand-side relaxation of the Harris ratio test
constexpr double LP_GAP_REL = 1e-8;    // largest primal-dual gap of an accepted step (relative)
constexpr double LP_ROW_TOL = 1e-7;    // largest violation of an extra initial row by z* (x the box size)

// ---------------------------------------------------------------- double-double
// Error-free transformations (Knuth's TwoSum, Dekker's fast two-sum for
// |a| >= |b|, the FMA form of the exact product) and the double-double sum,
// product and quotient built from them.  The _rn intrinsics keep the
// compiler from contracting or reassociating the error terms.
struct dd {
    double h, l;
};
__device__ __forceinline__ dd two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    return {s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}
__device__ __forceinline__ dd fast_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd two_prod(double a, double b) {
    const double p = __dmul_rn(a, b);
    return {p, __fma_rn(a, b, -p)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = two_sum(a.h, b.h);
    const dd t = two_sum(a.l, b.l);
    s.l = __dadd_rn(s.l, t.h);
    s = fast_two_sum(s.h, s.l);
    s.l = __dadd_rn(s.l, t.l);
    return fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.h, b.h);
    p.l = __fma_rn(a.h, b.l, p.l);
    p.l = __fma_rn(a.l, b.h, p.l);
    return fast_two_sum(p.h, p.l);
}
__device__ __forceinline__ dd dd_div(dd a, dd b) {  // long division, three quotient digits
    const double q1 = __ddiv_rn(a.h, b.h);
    dd r = dd_add(a, dd_neg(dd_mul({q1, 0.0}, b)));
    const double q2 = __ddiv_rn(r.h, b.h);
    r = dd_add(r, dd_neg(dd_mul({q2, 0.0}, b)));
    const double q3 = __ddiv_rn(r.h, b.h);
    return dd_add(fast_two_sum(q1, q2), {q3, 0.0});
}
__device__ __forceinline__ double dd_val(dd a) { return a.h + a.l; }

// The tableau: (d + 1) rows of W entries, hi and lo parts apart.
struct Tab {
    double* h;
    double* l;
    int W;
    __device__ dd at(int r, int c) const { return {h[(size_t)r * W + c], l[(size_t)r * W + c]}; }
    __device__ double hi(int r, int c) const { return h[(size_t)r * W + c]; }
    __device__ void set(int r, int c, dd x) const {
        h[(size_t)r * W + c] = x.h;
        l[(size_t)r * W + c] = x.l;
    }
};

struct LpArgs {
    const double* basis;  // [j][r][k], i x o x S
    int i, o, S;
    const double* U;      // qu x o, rows of unit norm
    const double* v;      // qu
    int qu;
    const double* Iz;     // qi x i
    const double* iota;   // qi
    int qi;
    const double* zlo;    // i (device, from the problem)
    const double* zhi;
    int m;                // primal constraints = dual columns
    int W;                // tableau row stride: m + d + 1
    int max_iter;         // per phase
    double* margin;       // S
    int* status;          // S
    double* zx;           // S x i
    double* yx;           // S x o
    int zonly;            // 1: the initial-set emptiness check (one CTA; the unsafe row is t >= 0)
    int* zflag;           // written by the check: 0 non-empty, 1 empty, 2 undecided; read by the steps
};

struct LpShared {
    int enter, leave, degen;
    dd piv;
};

// Pivot on row kp, column e: row kp /= T[kp][e], then every other row
// (the objective row d included) loses its multiple of row kp.
__device__ void lp_pivot(const Tab& T, int* bas, dd* fcol, int d, int kp, int e, LpShared& sh) {
    const int W = T.W;
    if (threadIdx.x == 0) sh.piv = T.at(kp, e);
    __syncthreads();
    for (int c = threadIdx.x; c < W; c += LNT) T.set(kp, c, c == e ? dd{1.0, 0.0} : dd_div(T.at(kp, c), sh.piv));
    for (int r = threadIdx.x; r <= d; r += LNT) fcol[r] = r == kp ? dd{0.0, 0.0} : T.at(r, e);
    __syncthreads();
    for (int idx = threadIdx.x; idx < (d + 1) * W; idx += LNT) {
        const int r = idx / W, c = idx - r * W;
        if (r == kp || (fcol[r].h == 0.0 && fcol[r].l == 0.0)) continue;
        T.set(r, c, c == e ? dd{0.0, 0.0} : dd_add(T.at(r, c), dd_neg(dd_mul(fcol[r], T.at(kp, c)))));
    }
    if (threadIdx.x == 0) bas[kp] = e;
    __syncthreads();
}

// One simplex phase over the entering columns [0, m) (artificial columns
// never enter).  Returns 0 optimal, 1 unbounded, 2 iteration limit.
//
// Pricing: the most negative reduced cost (Dantzig), ratio test: Harris's
// two passes (the smallest ratio with the right-hand sides relaxed by
// LP_HARRIS, then the largest pivot among the rows within it) -- few pivots
// and no tiny pivots.  After more than d degenerate pivots in a row the
// phase switches to Bland's rule (smallest entering index, smallest basic
// index among the tied rows whose pivot is not tiny) until a pivot makes
// progress, which rules out cycling.  Decisions use the hi parts.
__device__ int lp_phase(const Tab& T, int* bas, dd* fcol, int d, int m, double eps_rc, int max_iter,
                        LpShared& sh) {
    const int rhs = m + d;
    __shared__ double wval[LNT / 32];
    __shared__ int widx[LNT / 32];
    if (threadIdx.x == 0) sh.degen = 0;
    __syncthreads();
    for (int it = 0;; ++it) {
        const bool bland = sh.degen > d;  // uniform: read after a barrier
        // entering column: (reduced cost, index) minimum, or the first negative one
        double bv = -eps_rc;
        int bi = INT_MAX;
        for (int c = threadIdx.x; c < m; c += LNT) {
            const double x = T.hi(d, c);
            if (x < -eps_rc && (bland ? c < bi : (x < bv || (x == bv && c < bi)))) {
                bv = x;
                bi = c;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (bland ? oi < bi : (ov < bv || (ov == bv && oi < bi))) {
                bv = ov;
                bi = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            wval[threadIdx.x >> 5] = bv;
            widx[threadIdx.x >> 5] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < LNT / 32; ++w)
                if (bland ? widx[w] < bi : (wval[w] < bv || (wval[w] == bv && widx[w] < bi))) {
                    bv = wval[w];
                    bi = widx[w];
                }
            sh.enter = bi;
        }
        __syncthreads();
        const int e = sh.enter;
        if (e == INT_MAX) return 0;
        if (it >= max_iter) return 2;
        if (threadIdx.x < 32) {  // ratio test, warp 0
            const int lane = threadIdx.x;
            double q = INFINITY;
            for (int r = lane; r < d; r += 32) {
                const double a = T.hi(r, e);
                if (a > LP_EPS_PIV) q = fmin(q, (fmax(T.hi(r, rhs), 0.0) + (bland ? 0.0 : LP_HARRIS)) / a);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q = fmin(q, __shfl_xor_sync(0xffffffffu, q, o));
            const double qtie = bland ? q + 1e-12 * (1.0 + q) : q;
            double amax = 0.0;
            for (int r = lane; r < d; r += 32) {
                const double a = T.hi(r, e);
                if (a > LP_EPS_PIV && fmax(T.hi(r, rhs), 0.0) / a <= qtie) amax = fmax(amax, a);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            // Harris: the largest pivot (smallest row on ties); Bland: the
            // smallest basic index among pivots not tiny next to the largest
            int best = INT_MAX, brow = -1;
            for (int r = lane; r < d; r += 32) {
                const double a = T.hi(r, e);
                if (!(a > LP_EPS_PIV) || fmax(T.hi(r, rhs), 0.0) / a > qtie) continue;
                const int key = bland ? (a >= 1e-3 * amax ? bas[r] : INT_MAX) : (a == amax ? r : INT_MAX);
                if (key < best) {
                    best = key;
                    brow = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int orow = __shfl_xor_sync(0xffffffffu, brow, o);
                if (ob < best) {
                    best = ob;
                    brow = orow;
                }
            }
            if (lane == 0) {
                sh.leave = q == INFINITY ? -1 : brow;
                if (brow >= 0) {
                    const double step = fmax(T.hi(brow, rhs), 0.0) / T.hi(brow, e);
                    sh.degen = step <= 1e-12 ? sh.degen + 1 : 0;
                }
            }
        }
        __syncthreads();
        if (sh.leave < 0) return 1;
        lp_pivot(T, bas, fcol, d, sh.leave, e, sh);
    }
}

__global__ void __launch_bounds__(LNT) k_step_lp(LpArgs a) {
    extern __shared__ double smem[];
    __shared__ LpShared sh;
    const int d = a.i + 1, m = a.m, W = a.W, rhs = m + d, k = blockIdx.x;
    if (!a.zonly && *a.zflag != 0) {  // empty (or undecided) initial set: no step LP
        const int st = *a.zflag == 1 ? 2 : 1;
        if (threadIdx.x == 0) {
            a.status[k] = st;
            a.margin[k] = NAN;
        }
        for (int j = threadIdx.x; j < a.i; j += LNT) a.zx[(size_t)k * a.i + j] = NAN;
        for (int r = threadIdx.x; r < a.o; r += LNT) a.yx[(size_t)k * a.o + r] = NAN;
        return;
    }
    const size_t NT = (size_t)(d + 1) * W;
    const Tab T{smem, smem + NT, W};         // row d is the objective
    dd* cost = (dd*)(smem + 2 * NT);         // m: b of the dual (scaled)
    dd* fcol = cost + m;                     // d + 1
    int* bas = (int*)(fcol + d + 1);         // d
    // primal constraint columns, unscaled: A[col][row] with row = z_0..z_{i-1}, t
    const int nbox0 = a.qu + a.qi;
    for (size_t idx = threadIdx.x; idx < 2 * NT; idx += LNT) smem[idx] = 0.0;
    for (int c = threadIdx.x; c < m; c += LNT) cost[c] = {0.0, 0.0};
    __syncthreads();
    for (int idx = threadIdx.x; idx < (a.zonly ? 0 : a.qu * a.i); idx += LNT) {  // U_u B_k e_j
        const int u = idx / a.i, j = idx - u * a.i;
        double s = 0.0;
        for (int r = 0; r < a.o; ++r) s = fma(a.U[(size_t)u * a.o + r], a.basis[((size_t)j * a.o + r) * a.S + k], s);
        T.h[(size_t)j * W + u] = s;
    }
    for (int u = threadIdx.x; u < a.qu; u += LNT) {
        T.h[(size_t)a.i * W + u] = -1.0;  // the t coefficient
        cost[u] = {a.zonly ? 0.0 : a.v[u], 0.0};
    }
    for (int idx = threadIdx.x; idx < a.qi * a.i; idx += LNT) {
        const int q = idx / a.i, j = idx - q * a.i;
        T.h[(size_t)j * W + a.qu + q] = a.Iz[(size_t)q * a.i + j];
    }
    for (int q = threadIdx.x; q < a.qi; q += LNT) cost[a.qu + q] = {a.iota[q], 0.0};
    if (threadIdx.x == 0) {  // finite box sides, in column order
        int c = nbox0;
        for (int j = 0; j < a.i; ++j) {
            if (isfinite(a.zhi[j])) {
                T.h[(size_t)j * W + c] = 1.0;
                cost[c++] = {a.zhi[j], 0.0};
            }
            if (isfinite(a.zlo[j])) {
                T.h[(size_t)j * W + c] = -1.0;
                cost[c++] = {-a.zlo[j], 0.0};
            }
        }
    }
    __syncthreads();
    // unit-norm columns (exact double-double products of the double data and
    // the double scale); the t row is negated so that the right-hand side
    // -c = -e_t becomes +1 (all right-hand sides >= 0); artificial identity;
    // phase-1 objective: minimise the sum of the artificials
    for (int c = threadIdx.x; c < m; c += LNT) {
        double nrm = 0.0;
        for (int r = 0; r < d; ++r) nrm = fma(T.hi(r, c), T.hi(r, c), nrm);
        nrm = sqrt(nrm);
        const double sc = nrm > 0.0 ? 1.0 / nrm : 1.0;
        dd colsum{0.0, 0.0};
        for (int r = 0; r < d; ++r) {
            const dd x = two_prod(T.hi(r, c) * (r == a.i ? -1.0 : 1.0), sc);
            T.set(r, c, x);
            colsum = dd_add(colsum, x);
        }
        cost[c] = two_prod(cost[c].h, sc);
        T.set(d, c, dd_neg(colsum));
    }
    for (int r = threadIdx.x; r < d; r += LNT) {
        T.set(r, m + r, {1.0, 0.0});
        T.set(r, rhs, {r == a.i ? 1.0 : 0.0, 0.0});
        bas[r] = m + r;
    }
    if (threadIdx.x == 0) T.set(d, rhs, {-1.0, 0.0});
    __syncthreads();

    int st = 0;  // KV_LP_OPTIMAL
    // phase 1 is bounded below by 0: a column without a pivot there is rounding
    // noise in its reduced cost, and the sum of artificials decides
    int rc = lp_phase(T, bas, fcol, d, m, LP_EPS_RC, a.max_iter, sh);
    if (rc == 2) st = 3;                                  // KV_LP_ITER
    else if (-dd_val(T.at(d, rhs)) > LP_EPS_FEAS) st = 1;  // KV_LP_FAILED
    if (st == 0) {
        // basic artificials at level zero leave the basis where a structural
        // column can replace them (else their row is redundant)
        for (int r = 0; r < d; ++r) {
            if (bas[r] < m) continue;  // uniform: bas is shared
            if (threadIdx.x == 0) sh.enter = INT_MAX;
            __syncthreads();
            for (int c = threadIdx.x; c < m; c += LNT)
                if (fabs(T.hi(r, c)) > 1e-9) {
                    atomicMin(&sh.enter, c);
                    break;
                }
            __syncthreads();
            if (sh.enter != INT_MAX) lp_pivot(T, bas, fcol, d, r, sh.enter, sh);
        }
        // phase 2: the dual's costs, reduced against the current basis
        double cmax = 0.0;
        for (int c = 0; c < m; ++c) cmax = fmax(cmax, fabs(cost[c].h));
        for (int c = threadIdx.x; c < W; c += LNT) {
            dd x = c < m ? cost[c] : dd{0.0, 0.0};
            for (int r = 0; r < d; ++r) {
                const int bc = bas[r];
                if (bc < m) x = dd_add(x, dd_neg(dd_mul(cost[bc], T.at(r, c))));
            }
            T.set(d, c, x);
        }
        __syncthreads();
        rc = lp_phase(T, bas, fcol, d, m, LP_EPS_RC * fmax(1.0, cmax), a.max_iter, sh);
        if (rc == 1) st = 2;       // dual unbounded: the initial set is empty
        else if (rc == 2) st = 3;
    }
    if (a.zonly) {  // the check LP is bounded (t >= 0): unbounded dual = empty set
        if (threadIdx.x == 0) *a.zflag = st == 0 ? 0 : (st == 2 ? 1 : 2);
        return;
    }
    // z*_j: the multiplier of row z_j (sign +1), clamped into the box -- where
    // B_k is tiny next to the t coefficient two nearly parallel unsafe
    // columns can share the optimal basis and leave z* off the box by the
    // rounding of that ill-conditioned solve (the margin is unaffected)
    double* zs = (double*)fcol;  // free now: 2 (d + 1) >= i doubles
    __syncthreads();
    for (int j = threadIdx.x; j < a.i; j += LNT)
        zs[j] = st == 0 ? fmin(fmax(-dd_val(T.at(d, m + j)), a.zlo[j]), a.zhi[j]) : NAN;
    __syncthreads();
    // y* = B_k z*; the tableau's first row is free now
    double* ys = T.h;
    for (int r = threadIdx.x; r < a.o; r += LNT) {
        double y = 0.0;
        for (int j = 0; j < a.i; ++j) y = fma(a.basis[((size_t)j * a.o + r) * a.S + k], zs[j], y);
        a.yx[(size_t)k * a.o + r] = y;
        if (r < W) ys[r] = y;
    }
    for (int j = threadIdx.x; j < a.i; j += LNT) a.zx[(size_t)k * a.i + j] = zs[j];
    __syncthreads();
    // The margin is the primal objective at z*, max_u (U_u y* - upsilon_u):
    // the value the reported counter-example attains.  The step checks
    // itself: that value must equal the dual objective (no duality gap) and
    // z* must meet the extra initial rows; otherwise rounding has spoilt the
    // tableau and the step reports KV_LP_FAILED.
    if (threadIdx.x == 0) {
        double t = -INFINITY;
        for (int u = 0; u < a.qu; ++u) {
            double s = -a.v[u];
            for (int r = 0; r < a.o; ++r) s = fma(a.U[(size_t)u * a.o + r], r < W ? ys[r] : a.yx[(size_t)k * a.o + r], s);
            t = fmax(t, s);
        }
        if (st == 0) {
            const double gap = fabs(t - dd_val(T.at(d, rhs)));
            double zmax = 1.0;
            for (int j = 0; j < a.i; ++j) zmax = fmax(zmax, fmax(fabs(a.zlo[j]), fabs(a.zhi[j])));
            double viol = 0.0;
            for (int q = 0; q < a.qi; ++q) {
                double s = -a.iota[q], nq = 0.0;
                for (int j = 0; j < a.i; ++j) {
                    s = fma(a.Iz[(size_t)q * a.i + j], zs[j], s);
                    nq = fma(a.Iz[(size_t)q * a.i + j], a.Iz[(size_t)q * a.i + j], nq);
                }
                if (nq > 0.0) viol = fmax(viol, s / sqrt(nq));
            }
            if (gap > LP_GAP_REL * fmax(1.0, fabs(t)) || viol > LP_ROW_TOL * zmax) st = 1;
        }
        a.status[k] = st;
        a.margin[k] = st == 0 ? t : NAN;
    }
}

size_t lp_smem_bytes(int i, int m) {
    const size_t d = (size_t)i + 1, W = (size_t)m + d + 1;
    return (2 * (d + 1) * W + 2 * ((size_t)m + d + 1)) * sizeof(double) + d * sizeof(int);
}

// Two launches: the emptiness check of the initial set (one CTA; the unsafe
// part replaced by the single row t >= 0, so that its LP is bounded exactly
// when the set is non-empty), then one CTA per step.  With a non-empty
// initial set every step's LP is feasible and bounded (finite boxes).
int launch_step_lp(const Prob* p, const double* dU, const double* dv, int qu, const double* dIz,
                   const double* diota, int qi, int m, double* dmargin, int* dstatus, double* dzx, double* dyx,
                   int* dzflag) {
    LpArgs a{p->d_basis, p->i, p->o, p->steps + 1, dU, dv, qu, dIz, diota, qi, p->d_zlo, p->d_zhi, m,
             m + p->i + 2, 50 * (m + p->i + 1) + 100, dmargin, dstatus, dzx, dyx, 1, dzflag};
    const size_t sm = lp_smem_bytes(p->i, m);
    if (sm > 48 * 1024)
        KV_CHECK_CUDA(cudaFuncSetAttribute(k_step_lp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    LpArgs z = a;  // the check: one unsafe row (0 . z - t <= 0)
    z.qu = 1;
    z.m = 1 + qi + 2 * p->i;
    z.W = z.m + p->i + 2;
    z.max_iter = 50 * (z.m + p->i + 1) + 100;
    k_step_lp<<<1, LNT, lp_smem_bytes(p->i, z.m), p->ctx->stream>>>(z);
    KV_CHECK_CUDA(cudaGetLastError());
    a.zonly = 0;
    k_step_lp<<<(unsigned)(p->steps + 1), LNT, sm, p->ctx->stream>>>(a);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

}  // namespace kv
