/*
 * kv.h -- C ABI of libkv, a GB300 (sm_103a) library for the projected Krylov
 * safety check of affine systems x' = A x + b from "Numerical Verification of
 * Affine Systems with up to a Billion Dimensions" (Bak, Tran, Johnson).
 *
 * What one problem computes (all on the GPU):
 *   1. b is folded into the dynamics by a constant-1 variable: A' = [[A, b],
 *      [0, 0]] (Sec. 2.1).  Columns that carry the constant (is_fixed) run on
 *      A'; the others run on A.
 *   2. For every column E_j of the initial-space matrix (Sec. 3.2, x0 = E z):
 *      a Krylov simulation from v = E_j / ||E_j|| -- Lanczos for symmetric A
 *      (Alg. 3), Arnoldi otherwise (Alg. 1) -- with the output projection
 *      P = C V taken inside the loop so the basis is never stored for Lanczos
 *      (Alg. 4, Sec. 4.3).
 *   3. The basis matrix C e^{A t_k} E_j ~ ||E_j|| P e^{H t_k} e_1 for every
 *      step t_k = k dt, k = 0..steps (Eq. approx-formula, Sec. 4.2), with a
 *      batched FP64 scaling-and-squaring exponential of H (Pade-13 in shared
 *      memory up to dimension 64; above it, and for KV_EXPM_PROPAGATE, a
 *      degree-18 Taylor sum in global-memory GEMMs: the same e^{tH} up to
 *      rounding).
 *   4. Per step and output row r, the interval [lo, hi] of y_r = C_r x over
 *      the box z_j in [zlo_j, zhi_j], the first step whose upper bound reaches
 *      the unsafe half-space y_r >= theta_r, and the maximising box vertex as
 *      counter-example (the per-step LP of Sec. 2.1, solved in closed form for
 *      a box and one half-space per row).
 *
 * Conventions for every entry point:
 *   - Return value: KV_OK (0) or a KV_E* code; no exception crosses the ABI.
 *     kv_last_error() returns a message for the calling thread's last error.
 *   - Host pointers are read during the call only (copied to the device);
 *     the caller keeps ownership.  Pointers documented as device pointers are
 *     borrowed for the duration of the call.
 *   - Objects (kv_ctx, kv_sys, kv_prob) are owned by the caller and freed
 *     with the matching *_destroy.  A system must outlive its problems; a
 *     context must outlive everything created from it.
 *   - A kv_ctx is not thread-safe: use one per host thread.
 *   - Device memory comes from the context's pool (an arena over one device
 *     buffer); an allocation beyond it fails with KV_ENOMEM, never by trying
 *     the device allocator until it fails.
 *   - Index layout of grid systems: x fastest, idx = (z*ny + y)*nx + x.
 */
#ifndef KV_H
#define KV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define KV_OK 0
#define KV_EINVAL 1     /* bad argument (sizes, indices, flags, malformed CSR) */
#define KV_ENOMEM 2     /* the context's device pool cannot hold the request */
#define KV_ECUDA 3      /* a CUDA runtime call failed */
#define KV_ETIMEOUT 4   /* a device-side wait gave up (status word set by the kernel) */
#define KV_EBUSY 5      /* no free serving slot */
#define KV_ENOTREADY 6  /* a submitted problem has not finished */

/* storage precision of A's values and the Krylov vectors */
#define KV_FP64 0       /* IEEE double storage and arithmetic */
#define KV_FP32 1       /* float storage and stencil/SpMV arithmetic; every dot
                           product and norm is accumulated error-free in float
                           pairs and summed in double; H, the exponential and
                           the bounds are double */

#define KV_PREC_AUTO 2  /* kv_problem / kv_problem_bytes: KV_FP64 when the operator is
                           symmetric and its largest-eigenvalue bound mu (the one of the
                           error control) gives mu * steps * dt > -1 -- its slowest
                           mode loses less than a factor e over the horizon, so FP32
                           rounding of the stored Krylov vectors reaches the last
                           outputs undamped (an insulated heat model: measured
                           1.2e-6 .. 2.4e-6 with FP32 storage against the FP64 oracle)
                           -- else KV_FP32.  CSR systems keep their value precision;
                           KV_EINVAL when the rule asks for FP64 and the values are
                           FP32.  kv_problem_precision reports the choice. */

/* Krylov method */
#define KV_AUTO 0       /* Lanczos when the system is symmetric and the column
                           does not carry the constant variable, else Arnoldi */
#define KV_LANCZOS 1
#define KV_ARNOLDI 2

/* initial-space column kinds */
#define KV_COL_BOX 0    /* value on the grid box box_lo <= idx < box_hi */
#define KV_COL_SPARSE 1 /* (idx[e], val[e]) host arrays of nnz entries */
#define KV_COL_DENSE 2  /* host array of n entries */

/* how e^{H t_k} e_1 is formed for k = 0..steps */
#define KV_EXPM_PER_STEP 0   /* one Pade-13 scaling-and-squaring exponential per step */
#define KV_EXPM_PROPAGATE 1  /* M = e^{H dt} once, then u_k = M u_{k-1} */

typedef struct kv_ctx kv_ctx;
typedef struct kv_sys kv_sys;
typedef struct kv_prob kv_prob;

/* One column E_j of the initial-space matrix, with its box z_j in [zlo, zhi]
 * (Sec. 3.2).  is_fixed: z_j = 1 (zlo = zhi = 1 required) and the column
 * carries the constant-1 variable that folds b into the dynamics (Sec. 2.1,
 * "fixed" initial values, Fig. 2(c)). */
typedef struct {
    int32_t kind;           /* KV_COL_* */
    int32_t is_fixed;       /* 0 or 1 */
    double zlo, zhi;        /* zlo <= zhi */
    int64_t box_lo[3];      /* BOX: inclusive lower corner (x, y, z) */
    int64_t box_hi[3];      /* BOX: exclusive upper corner */
    double value;           /* BOX: value of E_j on the box */
    int64_t nnz;            /* SPARSE: entries */
    const int64_t *idx;     /* SPARSE: host, distinct, in [0, n) */
    const double *val;      /* SPARSE: host */
    const double *dense;    /* DENSE: host, n entries */
} kv_column;

/* A verification problem over one system (Sec. 2): initial set E z with a
 * box on z, outputs y = C x with C in CSR form over the n state variables
 * (Sec. 3.1), unsafe set y_r >= theta_r (theta_r = +inf: row not checked),
 * step dt and steps + 1 check points t_k = k dt (k = 0 included), Krylov
 * dimension krylov_m (the paper's k; 1 <= krylov_m <= KV_MAX_M, or
 * <= KV_MAX_M_LANCZOS when every column runs Lanczos).
 *
 * err_target > 0 turns on the a-posteriori error control of Alg. 2 / Alg. 4:
 * krylov_m is then the largest dimension, and each column stops at the first
 * of the dimensions 4, ceil(1.1 k), ... (the growth rule evaluated in IEEE
 * double) below krylov_m whose Lemma-1 bound (Sec. 4.2) is below err_target;
 * a column whose bound never gets there runs to krylov_m.  The bound is
 *   h_{k+1,k} e^{max(mu,0) T} sum_{j=1..steps} dt (|h(t_{j-1})| + |h(t_j)|) / 2,
 *   h(t) = (e^{t H_k})_{k,1},  T = steps dt,
 * the lemma applied with B = -A and its integral taken by the trapezoid rule
 * on the output grid; mu is an upper bound of the largest eigenvalue of
 * (A + A^T)/2 for the matrix the column works on (grid: the exact value;
 * CSR: the Gershgorin bound of the symmetric part, of A' = [[A, b], [0, 0]]
 * for a column that carries the constant).  err_target <= 0: fixed krylov_m.
 * The bound at the dimension used is reported either way (kv_result.err_bound). */
typedef struct {
    int32_t i;                  /* number of columns, >= 1 */
    const kv_column *cols;      /* host, i entries */
    int32_t o;                  /* number of output rows, >= 1 */
    const int64_t *c_row_ptr;   /* host, o+1 */
    const int64_t *c_col;       /* host, c_row_ptr[o] entries in [0, n) */
    const double *c_val;        /* host */
    const double *theta;        /* host, o */
    double dt;                  /* > 0 */
    int32_t steps;              /* >= 0 */
    int32_t krylov_m;
    int32_t method;             /* KV_AUTO | KV_LANCZOS | KV_ARNOLDI */
    int32_t expm_mode;          /* KV_EXPM_PER_STEP | KV_EXPM_PROPAGATE */
    int32_t batched;            /* CSR: 1 = all Arnoldi columns share one SpMM */
    int32_t flags;              /* KV_FLAG_* bits, 0 = defaults */
    double err_target;          /* > 0: error control with krylov_m as the largest dimension */
    int32_t simulate;           /* KV_SIM_FORWARD | KV_SIM_TRANSPOSE | KV_SIM_AUTO */
} kv_problem_desc;

/* kv_problem_desc.simulate: how the basis matrix C e^{At} E is built (Sec. 4.1).
 * FORWARD: one Krylov run per column of E (i runs), projected by C.
 * TRANSPOSE: one run per row of C of the transpose dynamics x' = A^T x
 *   (A'^T = [[A^T, 0], [b^T, 0]] when a column carries the constant), started
 *   at C_r^T and projected by E^T: C e^{At} E = (E^T e^{A^T t} C^T)^T, o runs.
 *   The per-run results of kv_result (H, P, beta0, m_used, err_bound) then
 *   have o entries, and P is i x krylov_m per run (E^T V).
 * AUTO: TRANSPOSE when o < i, else FORWARD (the smaller of i and o runs). */
#define KV_SIM_FORWARD 0
#define KV_SIM_TRANSPOSE 1
#define KV_SIM_AUTO 2

/* kv_problem_desc.flags */
#define KV_FLAG_TWO_PASS 1      /* grid Lanczos: use the two-pass kernels even where
                                   the single-pass TMA iteration applies */
#define KV_FLAG_NO_SPMM 2       /* CSR Arnoldi: one SpMV per column instead of the
                                   grouped SpMM (matrix read once per group) */
#define KV_FLAG_NO_AUTOTUNE 4   /* CSR Arnoldi: fixed SpMM shape instead of timing the
                                   candidates at kv_problem (and the on-disk cache) */
/* CSR Arnoldi SpMM shapes.  Column-major: G in {1, 2, 4, 8} columns share one
   read of the matrix and gather x_k[col] from each column's own vector.
   Interleaved: before each SpMM the group's current vectors are copied
   row-interleaved (row r holds x_0[r] .. x_{G-1}[r]), so one gather serves the
   G columns; G * element size in {16, 32, 64} bytes.  The autotuner times both
   forms (problems from 65536 rows) and keeps the fastest.  LPR lanes share a
   row: 1, 2 or 4 (column-major form), 0 (one lane per row, the warp's entries
   staged in shared memory by coalesced loads), 1 or 2 (interleaved form).
   The environment variable KV_SPMM_SHAPE="G,LPR" (G < 0 for the interleaved
   form of -G columns) fixes the shape of problems created while it is set;
   an unknown shape is ignored.  The interleaved form adds
   ceil(run / G) * G * N * element size bytes to kv_problem_bytes (run = the
   longest run of Arnoldi columns). */

/* Other environment variables the library reads (once per process):
   KV_AUTOTUNE_CACHE  path of the SpMM autotuner's cache file (default
                      $HOME/.cache/kv_autotune.txt);
   KV_PDL=0           launches the CSR Lanczos pair and the single-pass FP64
                      grid iteration without programmatic dependent launch
                      (the results are bit-identical);
   KV_FUSED64_UNIT=0  keeps every single-pass FP64 grid iteration in the plain
                      form, w stored as such, instead of the unit form that
                      stores w / (s_j coef/h_x^2) with one FP64 instruction a
                      point fewer (the results agree to rounding). */

#define KV_MAX_M 256           /* largest krylov_m when any column runs Arnoldi */
#define KV_MAX_M_LANCZOS 4096  /* largest krylov_m when every column runs Lanczos
                                  (above 64 the exponential runs in global memory) */

/* Results copied to the host.  lo and hi are required; every other array is
 * optional (NULL = not copied).  Layouts are row-major:
 *   lo, hi   o x (steps+1)                 [r][k]
 *   basis    i x o x (steps+1)             [j][r][k]: C e^{A t_k} E_j
 *   H        i x (krylov_m+1) x krylov_m   [j][row][col], Hessenberg /
 *                                          tridiagonal, the extra row kept
 *   P        i x o x krylov_m              [j][r][l] = C v_l
 *   beta0    i                             ||E_j|| (with the constant entry)
 *   m_used   i                             valid columns of H and P
 *   z_star   i                             counter-example z (unsafe only)
 *   err_bound i                            Lemma-1 bound at m_used, for the
 *                                          normalised start vector E_j/||E_j||
 * H, P, beta0, m_used and err_bound are per Krylov run: i runs, or o runs
 * under the transpose dynamics (kv_problem_runs gives the count; P is then
 * i x krylov_m per run). */
typedef struct {
    double *lo;
    double *hi;
    double *basis;
    double *H;
    double *P;
    double *beta0;
    int32_t *m_used;
    double *z_star;
    int32_t first_violation_step;   /* -1: safe */
    int32_t violation_row;          /* -1: safe */
    double y_star;                  /* hi_r(k) at the violation */
    double *err_bound;
} kv_result;

/* Library version string (static storage). */
const char *kv_version(void);

/* Message of the calling thread's last failed call ("" if none). */
const char *kv_last_error(void);

/* Create a context on CUDA device `device`.  pool: a device buffer of
 * pool_bytes the context sub-allocates from (borrowed until kv_destroy; must
 * be 256-byte aligned), or NULL to let the context allocate pool_bytes itself
 * once.  stream: a cudaStream_t to launch on, or NULL for a stream the
 * context creates.  Errors: KV_EINVAL, KV_ENOMEM, KV_ECUDA. */
int kv_create(kv_ctx **ctx, int device, void *pool, size_t pool_bytes, void *stream);
int kv_destroy(kv_ctx *ctx);

/* Bytes of the pool in use and in total. */
int kv_pool_stats(const kv_ctx *ctx, size_t *in_use, size_t *total);

/* Matrix-free grid system: A = coef * discrete Laplacian with spacing h[a]
 * per axis and a Dirichlet-0 boundary (semi-finite-difference heat model,
 * Sec. 5.3).  ndim = 2 or 3; dims[ndim..2] are ignored; b: host, n entries,
 * or NULL.  The Laplacian is symmetric, so KV_AUTO picks Lanczos for columns
 * without the constant variable. */
int kv_system_stencil(kv_ctx *ctx, kv_sys **out, int ndim, const int64_t dims[3], double coef,
                      const double h[3], const double *b);

/* Matrix-free grid system with a coefficient per face of the grid box (the
 * boundary models of Sec. 5.3).  face: host, 2*ndim entries (x low, x high,
 * y low, y high[, z low, z high]), each finite and >= 0, or NULL for
 * Dirichlet-0 (then identical to kv_system_stencil).  A grid point p on face
 * f gets -face[f] v_p in place of the coupling coef/h_a^2 (v_q - v_p) to its
 * missing neighbour q:
 *     (A v)_p = sum over neighbours q in the grid of coef/h_a^2 (v_q - v_p)
 *               - sum over the faces f that p lies on of face[f] v_p.
 * face[f] = coef/h_a^2 is the Dirichlet-0 boundary of the vertex grid (the
 * ghost value 0), 0 an insulated face, and for the paper's heat model (unit
 * cube of N^3 cells, h = 1/N, insulated except x = 1 with heat exchange
 * constant g0 toward ambient 0) face[1] = g / h with
 * g = g0 (2 coef/h) / (2 coef/h + g0), the half cell between the last
 * cell's centre and the face eliminated.  A is symmetric, so KV_AUTO picks
 * Lanczos.  Face coefficients need coef > 0 (the kernels hold each as its
 * share face[f] / (coef/h_a^2) of the coupling it replaces).  Errors:
 * KV_EINVAL (bad sizes, face values, or a face array with coef <= 0),
 * KV_ENOMEM, KV_ECUDA. */
int kv_system_grid(kv_ctx *ctx, kv_sys **out, int ndim, const int64_t dims[3], double coef,
                   const double h[3], const double *face, const double *b);

/* Sparse system in CSR form (row_ptr n+1 int64 starting at 0 and
 * non-decreasing, col int32 in [0, n), strictly increasing within a row, val
 * doubles).  When on_device is 0 the three arrays are host memory and are
 * copied; when 1 they are device pointers copied device-to-device.  row_ptr is
 * checked on the host (device arrays: after one copy to the host); the column
 * indices are checked on the device after the copy, before any kernel reads
 * through them, and an error names the first offending entry in storage
 * order.  value_precision (KV_FP64 or KV_FP32) is the storage of the values
 * and must match the precision of the problems run on the system; KV_FP32
 * rounds each double to the nearest float on the device (host values pass
 * through a staging buffer of at most 32 MB from the pool).  Errors: KV_EINVAL (malformed arrays, out-of-range or unsorted
 * columns), KV_ENOMEM, KV_ECUDA.  symmetric: the caller's promise that A is
 * symmetric (enables Lanczos).  b: host, n entries, or NULL. */
int kv_system_csr(kv_ctx *ctx, kv_sys **out, int64_t n, const int64_t *row_ptr, const int32_t *col,
                  const double *val, const double *b, int symmetric, int value_precision,
                  int on_device);
int kv_sys_destroy(kv_sys *sys);

/* Create a problem on a system: validates the description, reserves its
 * device memory from the pool (KV_ENOMEM if it does not fit) and uploads the
 * initial-space columns and C.  precision: KV_FP64 or KV_FP32 storage of
 * the Krylov vectors. */
int kv_problem(kv_ctx *ctx, kv_prob **out, const kv_sys *sys, const kv_problem_desc *desc,
               int precision);
int kv_prob_destroy(kv_prob *prob);

/* Storage precision a problem runs in (KV_FP64 or KV_FP32; the choice made
 * for KV_PREC_AUTO). */
int kv_problem_precision(const kv_prob *prob, int32_t *precision);

/* Number of Krylov runs of a problem (i, or o with the transpose dynamics)
 * and whether the transpose dynamics run: the length of the per-run arrays of
 * kv_result. */
int kv_problem_runs(const kv_prob *prob, int32_t *runs, int32_t *transposed);

/* Device bytes kv_problem would reserve (the memory model of Sec. 4.2-4.3 for this
 * implementation: two n-vectors for Lanczos, m+1 for Arnoldi, plus the
 * o x i x (steps+1) basis of Eq. memory_basis and small state). */
int kv_problem_bytes(const kv_sys *sys, const kv_problem_desc *desc, int precision, size_t *bytes);

/* Enqueue the whole path on the context stream and return; results stay on
 * the device until kv_fetch. */
int kv_enqueue(kv_prob *prob);

/* Wait for the problem's work and copy its results to the host.  The results
 * are copied in every case; the status word the kernels set turns into the
 * return code: KV_ETIMEOUT (a bounded device wait expired), KV_EINVAL (an
 * index outside its vector was skipped by a device-side check; a Krylov
 * scalar was not finite, i.e. the system or the initial set holds a NaN or
 * overflows; or an exponential of H needed more scaling squarings than were
 * launched, i.e. ||dt H||_1 beyond 2^32 or beyond the operator's norm bound),
 * KV_ECUDA (a CUDA error). */
int kv_fetch(kv_prob *prob, kv_result *res);

/* kv_enqueue + kv_fetch. */
int kv_run(kv_prob *prob, kv_result *res);

/* Per-kernel timing with CUDA events on the context stream.  enable != 0
 * starts recording every launch (clearing earlier records); kv_profile_read
 * synchronises and reports, for the kernel family `name`, the number of
 * launches and their summed duration in milliseconds. */
int kv_profile_enable(kv_ctx *ctx, int enable);
int kv_profile_read(kv_ctx *ctx, const char *name, int64_t *launches, double *total_ms);

/* Number of kernel launches the context has issued since creation. */
int kv_launch_count(const kv_ctx *ctx, int64_t *launches);

/* ------------------------------------------------------- packed queries --
 * Many small problems under one CUDA graph.  A small query is dozens of tiny
 * kernels whose cost is launch latency; kv_graph_create records the whole
 * path of n problems (all created on ctx, any mix of systems) by stream
 * capture, with the problems on up to KV_GRAPH_BRANCHES parallel branches, and
 * kv_graph_launch replays everything with one graph launch on the context
 * stream.  After a launch each problem's results are read with kv_fetch, as
 * after kv_enqueue.  The graph holds the problems' device buffers: destroy it
 * before any of its problems, and do not enqueue those problems elsewhere
 * while a launch is in flight.  Per-kernel profiling must be off while
 * capturing.  Errors: KV_EINVAL, KV_ECUDA. */
#define KV_GRAPH_BRANCHES 8
typedef struct kv_graph kv_graph;
int kv_graph_create(kv_ctx *ctx, kv_prob *const *probs, int32_t n, kv_graph **out);
int kv_graph_launch(kv_graph *graph);
int kv_graph_destroy(kv_graph *graph);

/* ------------------------------------------------------------- serving --
 * Continuous batching of verification queries on one context.  The paper
 * verifies one problem at a time; the server keeps several on the device at
 * once.  A worker thread owned by the server admits queued queries in
 * arrival order whenever one of `slots` slots is free and the context pool
 * can hold the query's system and problem (device memory is reserved as in
 * kv_problem, the memory model of Sec. 4.2-4.3; a query that does not fit waits for
 * running ones to finish, and one that cannot fit an idle pool fails with
 * KV_ENOMEM).  Each admitted query's whole path is enqueued on its slot's own
 * stream, so the work of different queries overlaps on the device; on
 * completion its results are copied to host storage and its device memory
 * and slot are released.  Results are identical to kv_run on the same query
 * (deterministic reductions; queries share nothing but the read-only device
 * copy of a CSR system, below). */
typedef struct kv_server kv_server;

/* One query: a system (as for kv_system_stencil, kv_system_grid or kv_system_csr, host
 * arrays) and a problem description with its precision.  The kv_column array
 * is copied by kv_submit; every other host array the query references (CSR
 * arrays, b, face, column idx/val/dense arrays, C arrays, theta) must stay valid,
 * with unchanged contents, until kv_poll has returned something other than
 * KV_ENOTREADY for it.
 *
 * CSR queries that name the same row_ptr, col, val and b pointers with the
 * same n, symmetric and precision share one device copy of the system: it is
 * built (kv_system_csr: validation, upload, the log-norm bound) when the first
 * of them is admitted and released when the last of them queued or running
 * finishes, or earlier when the pool cannot hold an admission and no running
 * query uses it (it is then rebuilt for the next query naming it).  Equal
 * pointers are taken to mean equal contents, which the rule above guarantees
 * while any of the queries is unpolled.  A shared copy changes no result. */
typedef struct {
    int32_t kind;               /* 0: grid system, 1: CSR system */
    int32_t ndim;               /* grid: 2 or 3 */
    int64_t dims[3];            /* grid */
    double coef;                /* grid */
    double h[3];                /* grid */
    int64_t n;                  /* CSR */
    const int64_t *row_ptr;     /* CSR, host */
    const int32_t *col;         /* CSR, host */
    const double *val;          /* CSR, host */
    int32_t symmetric;          /* CSR */
    const double *b;            /* host, n entries, or NULL */
    kv_problem_desc desc;       /* the problem */
    int32_t precision;          /* KV_FP64 | KV_FP32 (CSR values stored likewise) */
    const double *face;         /* grid: host, 2 ndim face coefficients as for kv_system_grid,
                                   or NULL for the Dirichlet-0 boundary of kv_system_stencil */
} kv_query;

/* Start a server on ctx with `slots` concurrent queries (1..256).  While the
 * server exists the context belongs to its worker thread: make no other call
 * on ctx (or on objects created from it) until kv_server_destroy. */
int kv_server_create(kv_ctx *ctx, kv_server **out, int32_t slots);

/* Wait for every submitted query to finish, stop the worker, release the
 * server's streams.  Results not yet polled are discarded. */
int kv_server_destroy(kv_server *server);

/* Queue one query; returns its ticket.  Thread-safe.  Errors: KV_EINVAL,
 * KV_EBUSY (server shutting down). */
int kv_submit(kv_server *server, const kv_query *query, uint64_t *ticket);

/* KV_ENOTREADY while the query is queued or running.  Otherwise the query's
 * status (KV_OK or the error it failed with): on KV_OK its results are copied
 * into `res` (lo and hi required; beta0, m_used, z_star optional; basis, H, P
 * are not kept by the server) and latency_ms (optional) receives the time
 * from kv_submit to the results being on the host.  A ticket can be polled
 * to completion once.  Thread-safe. */
int kv_poll(kv_server *server, uint64_t ticket, kv_result *res, double *latency_ms);

/* Counters: queries admitted, completed, still queued, the largest number
 * running at once, and admissions deferred because the pool was full. */
int kv_server_stats(kv_server *server, int64_t *admitted, int64_t *completed, int64_t *pending,
                    int32_t *max_running, int64_t *memory_waits);

/* Shared CSR systems: device copies built, admissions that used a copy already
 * on the device, copies released early to make room, and copies on the device
 * now.  Any pointer may be NULL.  Thread-safe.  Errors: KV_EINVAL (NULL server). */
int kv_server_system_stats(kv_server *server, int64_t *built, int64_t *reused, int64_t *released,
                           int64_t *resident);

/* Polyhedral initial and unsafe sets (Sec. 2.1, over the projected basis of
 * Sec. 3.1-3.2).  The closed-form bounds of kv_run treat each output row as
 * its own half-space over a box of z; kv_check_polytope instead solves, at
 * every step k, the LP of Sec. 2.1 for an unsafe set given as a conjunction
 * U y <= upsilon of rows over the o outputs and an initial set given by the
 * columns' boxes and optional extra rows I z <= iota over the i columns:
 *     t*_k = min over the initial set of max_u (U_u B_k z - upsilon_u) / ||U_u||
 * with B_k = C e^{A t_k} E the o x i basis matrix.  t*_k <= 0 iff a state of
 * the initial set reaches the unsafe set at step k; for one unsafe row t*_k is
 * the signed distance (in output units) from the reachable output interval
 * to the half-space.  The LP's optimal value is unique; the minimiser z* (a
 * counter-example where t*_k <= tol) need not be. */
typedef struct {
    int32_t rows;        /* number of inequalities */
    const double *a;     /* host, rows x dim, row-major (dim = o for the unsafe set, i for the initial set) */
    const double *rhs;   /* host, rows */
} kv_polytope;

/* kv_lp_result.status per step */
#define KV_LP_OPTIMAL 0
#define KV_LP_FAILED 1     /* the dual's phase 1 found no feasible point (numerical failure) */
#define KV_LP_EMPTY 2      /* the initial set is empty */
#define KV_LP_ITER 3       /* iteration limit of a simplex phase reached */

typedef struct {
    double *margin;                /* caller, steps+1: t*_k (NaN unless KV_LP_OPTIMAL) */
    int32_t *status;               /* caller, steps+1: KV_LP_*; every step checks its own answer (no
                                      primal-dual gap, z* in the initial set) and reports KV_LP_FAILED
                                      where rounding has spoilt it */
    double *z;                     /* caller or NULL, (steps+1) x i: the minimiser per step */
    int32_t first_violation_step;  /* first k with KV_LP_OPTIMAL and margin <= tol, -1: none */
    double *z_star;                /* caller or NULL, i: the minimiser at that step */
    double *y_star;                /* caller or NULL, o: B_k z* at that step */
} kv_lp_result;

/* The per-step LPs for a problem whose results are complete (after kv_run, or
 * kv_enqueue + kv_fetch): one CTA per step on the device (dense two-phase
 * simplex on the LP's dual in shared memory, double-double tableau) over the basis
 * kept on the device, on the context's stream; the call waits for them.
 * unsafe: rows over the o outputs (rows >= 1, no zero row); init: rows over
 * the i columns or NULL; every column's box must be finite.  The LP must fit
 * one CTA's shared memory: 16 ((i+2)(m+i+2) + m + i + 2) + 4 (i+1) bytes with
 * m = unsafe rows + init rows + 2 i, at most the device's opt-in limit
 * (232448 bytes on GB300).  Temporary device memory (about 8 (steps+1)(i+o+2)
 * bytes) comes from the context's pool.  Errors: KV_EINVAL (bad argument, the
 * problem has not run, a set or LP too large), KV_ENOMEM, KV_ECUDA. */
int kv_check_polytope(kv_prob *prob, const kv_polytope *unsafe, const kv_polytope *init, double tol,
                      kv_lp_result *res);

/* Grid points the no-allocation entry point below can hold. */
#define KV_NOALLOC_MAX_N 262144

/* Projected Lanczos on a small grid without any device allocation.  The paper
 * has no counterpart: this exists for callers that cannot allocate device
 * memory when they need a result -- real-time or embedded hosts that reserve
 * all device memory up front and forbid allocation afterwards, callers running
 * inside another runtime's allocator or memory-pool callback, which must not
 * re-enter the driver's allocator.  It runs the FP64 two-pass grid Lanczos
 * iterations of kv_run for one box column (value on box_lo <= idx < box_hi) on
 * the grid of kv_system_stencil (Dirichlet-0, no forcing term) and writes H
 * ((krylov_m+1) x krylov_m, row-major), P (o x krylov_m: C v_l), beta0
 * (||E||) and m_used (valid columns) to the caller's device buffers.
 * krylov_m is in [1, KV_MAX_M]: the main path's larger Lanczos limit serves
 * its error control, which this entry point does not have.  C is given in
 * CSR form with device arrays: c_row_ptr holds o+1 offsets, c_col and c_val
 * hold c_row_ptr[o] entries each (the caller guarantees these lengths).  The
 * first kernel checks what it can: offsets that do not start at 0 or that
 * decrease, or a column index outside [0, n), end the call's work before
 * anything is read through them, with m_used = -1 and H, P zero.  All working
 * memory (two Krylov vectors, reduction partials, column state, about
 * 4.2 MB) lives in one fixed device array that every GPU loading the library
 * holds until exit; nothing is allocated or freed.  Grids with more than
 * KV_NOALLOC_MAX_N points are rejected with KV_EINVAL.  Work is enqueued on
 * `stream` (a cudaStream_t, NULL = default stream) and the call returns
 * without waiting.  The array is shared by all calls on a device and keeps
 * the last call's contents: calls whose work overlaps on the GPU race on it.
 * The first call on a device looks up the array's address on that device;
 * make that first call before any stream capture begins.  That address is
 * kept for the life of the process, so after cudaDeviceReset on a device this
 * entry point must not be called on it again.  The calling thread's current
 * device is the same after the call as before.  Errors: KV_EINVAL (NULL
 * argument, bad sizes), KV_ECUDA. */
int kv_grid_lanczos_noalloc(int device, void *stream, int ndim, const int64_t dims[3], double coef,
                            const double h[3], const int64_t box_lo[3], const int64_t box_hi[3], double value,
                            int32_t o, const int64_t *c_row_ptr, const int64_t *c_col, const double *c_val,
                            int32_t krylov_m, double *H, double *P, double *beta0, int32_t *m_used);

/* Check of the failure path of the device waits.  Not in the paper: the
 * single-pass grid kernel waits for its TMA stages on mbarriers with a limit
 * on the number of polls and reports an expired wait through the column's
 * status word (kv_fetch then returns KV_ETIMEOUT) instead of hanging the GPU.
 * This launches one block that waits, with the same bounded-wait routine and
 * `polls` polls (1 .. 4194304), on an mbarrier that nothing completes, so the
 * wait must expire; the block records the expiry in a status word and exits.
 * The call waits for the block and returns KV_ETIMEOUT when the wait expired
 * (the expected outcome), KV_OK if it did not, KV_EINVAL for a bad argument,
 * KV_ECUDA on a CUDA error.  The device and any context on it stay usable. */
int kv_diag_bounded_wait(int device, int64_t polls);

#ifdef KV_DEBUG
/* Debug build only (compiled with -DKV_DEBUG; not in the paper): overwrite
 * entry e of a forward problem's device copy of the output matrix's column
 * indices with `value`, which the host validation of kv_problem would have
 * refused, so that a test can check that the device-side bounds checks skip
 * such an index instead of reading through it (kv_fetch then returns
 * KV_EINVAL).  Waits for the context stream first.  Errors: KV_EINVAL (NULL
 * problem, a transposed problem, e outside C's entries), KV_ECUDA. */
int kv_debug_set_c_col(kv_prob *prob, int64_t e, int64_t value);
#endif

/* The device's FP64 instruction rate, measured.  Not in the paper: the FP64
 * grid iteration is bound by the FP64 pipe of this GPU (not by HBM), and its
 * roofline takes this rate as the peak.  Runs eight independent chains of
 * FP64 fused multiply-adds (then of FP64 additions) per thread on 8 blocks of
 * 256 threads per SM and reports operations per second (one FMA or add of
 * one thread = one operation) over the best of five timed launches.
 * Allocates a small device buffer and a stream for the call and waits for
 * them.  Errors: KV_EINVAL (NULL argument, bad device), KV_ECUDA. */
int kv_diag_fp64_rate(int device, double *fma_per_s, double *add_per_s);

#ifdef __cplusplus
}
#endif
#endif /* KV_H */
