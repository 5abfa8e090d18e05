// kv_internal.h -- host/device declarations shared by the libkv translation
// units (not part of the public ABI; see include/kv.h).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/kv.h"

namespace kv {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
#define KV_CHECK_CUDA(call)                                                        \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) {                                                   \
            ::kv::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), \
                            __FILE__, __LINE__);                                   \
            return KV_ECUDA;                                                       \
        }                                                                          \
    } while (0)

// Makes `device` current for the guard's scope and then makes the calling
// thread's previous current device current again, so no call of the library
// leaves the caller switched to another device.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != device) err = cudaSetDevice(device);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};
#define KV_WITH_DEVICE(dev)                                                                            \
    ::kv::DeviceGuard kv_device_guard_(dev);                                                          \
    if (kv_device_guard_.err != cudaSuccess) {                                                        \
        ::kv::set_error("cudaSetDevice(%d) failed: %s", (int)(dev), cudaGetErrorString(kv_device_guard_.err)); \
        return KV_ECUDA;                                                                               \
    }

// ------------------------------------------------------------------- arena
// First-fit allocator over one device buffer; 256-byte granularity.  All
// device memory of a context comes from here, so admission is a bookkeeping
// question (does the request fit?) rather than a cudaMalloc that may fail.
class Arena {
  public:
    void init(char* base, size_t size);
    // returns nullptr when the request does not fit
    void* alloc(size_t bytes);
    void free(void* p);
    size_t in_use() const { return in_use_; }
    size_t total() const { return size_; }
    size_t largest_free() const;

  private:
    char* base_ = nullptr;
    size_t size_ = 0, in_use_ = 0;
    std::map<size_t, size_t> free_;  // offset -> size
    std::map<size_t, size_t> used_;  // offset -> size
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* pool = nullptr;
    bool own_pool = false;
    Arena arena;
    int64_t launches = 0;
    bool profiling = false;
    bool capturing = false;  // inside kv_graph_create's stream capture
    struct Rec {
        std::string name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> spare_events;
};

// Programmatic dependent launch (griddepcontrol, sm_90 and later).  A kernel
// of a dependent chain (each reads what the one before it in the stream
// wrote) starts with dep_wait(), which returns once the previous kernel has
// completed and its writes are visible, then calls dep_release(), which lets
// the next kernel be launched as soon as every block of this one has
// started, so the next grid's launch and ramp overlap this grid's run instead
// of following its end.  Both are no-ops in a kernel launched without the
// attribute.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Whether a launch on the context's stream may carry the attribute: not
// while profiling (events between the launches) or capturing a graph, and
// not when the environment variable KV_PDL is 0.
bool dep_launch_ok(const Ctx* c);

// kern<<<grid, block, smem, s>>>(args...), with the programmatic-serialisation
// attribute when pdl (dep_launch_ok of the context, and no event or other
// stream work of the caller between this launch and the kernel before);
// kern must begin with dep_wait().
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    if (!pdl) {
        kern<<<grid, block, smem, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Records one launch: bumps the launch counter and, when profiling, brackets
// the launch with events on the context stream.
struct LaunchScope {
    LaunchScope(Ctx* c, const char* name);
    ~LaunchScope();
    Ctx* ctx;
    int rec = -1;
};

struct Sys {
    Ctx* ctx = nullptr;
    int kind = 0;  // 0 grid, 1 csr
    int ndim = 0;
    int64_t dims[3] = {1, 1, 1};
    double coef = 0, h[3] = {1, 1, 1};
    // grid boundary: gamma per face (x low, x high, y low, y high, z low, z
    // high); a point on face f gets -gamma_f v_p in place of the coupling to
    // the missing neighbour.  gamma = coef / h_a^2 on every face is the
    // Dirichlet-0 boundary (faces == false); axes beyond ndim have 0.
    double face[6] = {0, 0, 0, 0, 0, 0};
    bool faces = false;
    int64_t n = 0, nnz = 0;
    int64_t* d_rp = nullptr;
    int32_t* d_col = nullptr;
    void* d_val = nullptr;  // double or float
    int val_prec = KV_FP64;
    double* d_b = nullptr;
    bool symmetric = false;
    // upper bounds of the largest eigenvalue of (A + A^T)/2, for A and for
    // A' = [[A, b], [0, 0]] (Lemma 1 of Sec. 4.2 takes e^{max(mu,0) T})
    double mu = 0.0, mu_aug = 0.0;
    // a bound of ||A||_2 for a symmetric operator (Gershgorin: the largest
    // absolute row sum, rounded up), +inf where none is known; it bounds
    // ||H_k||_1 <= 3 ||A||_2 for the Lanczos H and so the squarings of its
    // exponential
    double norm2_bound = INFINITY;
    // A^T in CSR form (non-symmetric CSR only), built on first use by a
    // problem that runs the transpose dynamics (Sec. 4.1)
    int64_t* d_rpT = nullptr;
    int32_t* d_colT = nullptr;
    void* d_valT = nullptr;
};

// --------------------------------------------------------------- device state
// Per-column Krylov state kept on the device so the iteration needs no host
// round trip: the stored buffer holding v_j is scaled by s[j] on read (lazy
// normalisation), beta0 = ||E_j||, done = breakdown or zero column.
struct ColState {
    double beta0;
    int done;
    int m_used;
    int status;
    int pad;
    double s[KV_MAX_M_LANCZOS + 2];
};

struct CDesc {  // output matrix C in CSR form on the device
    int o;
    const int64_t* rp;
    const int64_t* col;
    const double* val;
    int64_t n;  // length of the vectors C is applied to (column indices lie in [0, n))
};

// ColState::status bits, reported by kv_fetch
constexpr int KV_ST_TIMEOUT = 1;    // a bounded device wait expired
constexpr int KV_ST_INDEX = 2;      // an index outside its vector was skipped, not read
constexpr int KV_ST_NONFINITE = 4;  // alpha or beta of an iteration is not finite
constexpr int KV_ST_SCALING = 8;    // an exponential needed more squarings than were launched

// One term of C_r . x: an entry whose column lies outside the vector is
// skipped (not read) and recorded in *status.
template <typename T>
__device__ __forceinline__ double c_entry(const CDesc& cd, int64_t e, const T* x, int* status) {
    const int64_t c = cd.col[e];
    if (c < 0 || c >= cd.n) {
        atomicOr(status, KV_ST_INDEX);
        return 0.0;
    }
    return cd.val[e] * (double)__ldcg(x + c);
}

struct Reduce {  // scratch of one deterministic grid reduction
    double* partials;
    unsigned* counter;
};

struct StencilGeom {
    int64_t nx, ny, nz;
    double kx, ky, kz, kc;  // kc = -2 (kx + ky + kz)
    // per face (x low, x high, y low, y high, z low, z high): rho = gamma /
    // kappa_axis, the share of the Dirichlet ghost coupling the face keeps
    // (1: Dirichlet-0, 0: insulated); the ghost value of the pair-sum form is
    // (1 - rho) v_p
    double rho[6];
};

struct Prob {
    Ctx* ctx = nullptr;
    const Sys* sys = nullptr;
    int prec = KV_FP64;
    int i = 0, o = 0, m = 0, steps = 0;
    double dt = 0;
    int expm_mode = KV_EXPM_PER_STEP;
    int batched = 0;
    int flags = 0;
    double err_target = 0.0;     // > 0: a-posteriori error control (Alg. 2 / Alg. 4)
    bool fused = false;          // single-pass TMA Lanczos iterations on the grid (FP32)
    bool fused64 = false;        // single-pass TMA Lanczos iterations on the grid (FP64)
    bool ran = false;            // enqueued at least once (the basis on the device is a result)
    std::vector<int> method;     // per column: KV_LANCZOS | KV_ARNOLDI
    std::vector<int> aug;        // per column: runs on A' (carries the constant)
    std::vector<kv_column> cols; // host copy (pointers cleared)
    std::vector<int64_t*> d_sidx;
    std::vector<int64_t> sidx_n;  // entries uploaded to d_sidx / d_sval (the scatter's count)
    std::vector<double*> d_sval;
    std::vector<double*> d_dense;
    // device arrays
    int64_t c_nnz = 0;  // entries of C (host copy of d_crp[o])
    int64_t* d_crp = nullptr;
    int64_t* d_ccol = nullptr;
    double* d_cval = nullptr;
    double* d_theta = nullptr;
    double* d_zlo = nullptr;
    double* d_zhi = nullptr;
    ColState* d_state = nullptr;
    double* d_H = nullptr;
    double* d_P = nullptr;
    double* d_basis = nullptr;
    double* d_lo = nullptr;
    double* d_hi = nullptr;
    double* d_zstar = nullptr;
    double* d_ystar = nullptr;
    int* d_viol = nullptr;
    double* d_err = nullptr;    // per column: Lemma-1 bound at the dimension used
    double* d_bpart = nullptr;  // column-chunk partial bounds (many columns only)
    double* d_hlast = nullptr;  // per column, steps+1: |(e^{t_k H} e_1)_mu|, the integrand of the bound
    double* d_lx = nullptr;     // scratch of the global-memory exponential (one batch of runs)
    // transpose dynamics (Sec. 4.1).  Outer problem: the basis matrix is built
    // from the runs of `inner` (one per output row, on A^T or A'^T, projected
    // by E'^T) and transposed; `view` is the operator the inner runs use.
    Prob* inner = nullptr;
    Sys* view = nullptr;
    // inner problem: runs of the transpose dynamics (the constant entry of a
    // start vector is 0, not 1); d_brow = b when the runs are on A'^T, whose
    // last row b . x is computed after each SpMV (k_row_dot)
    bool trans_runs = false;
    const double* d_brow = nullptr;
    double* d_rowdot = nullptr;  // i x row_dot_blocks() partials, then i tickets
    void* d_vec = nullptr;  // Krylov vectors
    int64_t N = 0;          // vector length (n, or n+1 if any column is augmented)
    int nvec = 0;           // vectors of length N per vector set
    int nsets = 1;          // vector sets (grid: 1, columns run in turn; CSR: one per column)
    unsigned* d_counters = nullptr;  // per-column reduction tickets (CSR)
    int* d_aug = nullptr;            // per-column: runs on A' (CSR)
    void* d_arnoldi = nullptr;       // per-column Gram matrix and coefficients (CSR)
    int spmm_G = 0, spmm_LPR = 0;    // CSR Arnoldi SpMM shape (autotuned; 0 = per-column SpMV;
                                     // G < 0: groups of -G columns read from d_xi)
    void* d_xi = nullptr;  // row-interleaved copy of the Arnoldi columns' current vectors
    Reduce red{};
    int red_slots = 0;
    std::vector<void*> allocs;
    cudaEvent_t done_ev = nullptr;
};

// ------------------------------------------------------------ launchers
// grid stencil (k_stencil.cu)
int stencil_blocks(const StencilGeom& g, int* zc);
int launch_stencil_init_box(Prob* p, int j, void* B);
int launch_stencil_alpha(Prob* p, int j, int it, const void* B);
int launch_stencil_update(Prob* p, int j, int it, const void* B, void* A);

// single-pass TMA Lanczos iteration, FP32 grids (k_stencil_tma.cu)
bool fused_tma_supported(const Prob* p);
int fused_tma_blocks(const Prob* p, int* zc);
int launch_lanczos_fused(Prob* p, int j, int it, const void* B, const void* A, void* W);

// single-pass TMA Lanczos iteration, FP64 grids (k_stencil_tma64.cu)
bool fused64_supported(const Prob* p);
int fused64_blocks(const Prob* p);
int fused64_prepare();
int launch_lanczos_fused64(Prob* p, int j, int it, const void* B, const void* Aprev, void* W);

// a-posteriori error bound (k_expm.cu): the exponentials of H_k at every
// step for columns j0 .. j0+ncols-1 (dim = k), then the bound and the stop
// decision; dim = 0: the bound at each column's m_used after the final basis
int launch_error_check(Prob* p, int j0, int ncols, int dim);
// Alg. 2 / Alg. 4: whether the error bound is evaluated after the iteration
// that completes Krylov dimension k (error control on, k in 4, ceil(1.1 k),
// ... in IEEE double, k < m)
inline bool is_checkpoint(const Prob* p, int k) {
    if (!(p->err_target > 0.0)) return false;
    for (int c = 4; c < p->m; c = (int)ceil(1.1 * (double)c))
        if (c == k) return true;
    return false;
}
int launch_error_final(Prob* p);
// Gershgorin bound of the symmetric part of a CSR matrix (k_lognorm.cu)
int csr_lognorm_bounds(Sys* s, const double* b_host, double* mu, double* mu_aug, double* row_abs_max);

// transpose dynamics (k_csr_transpose.cu)
int csr_build_transpose(Sys* s);
// k_csr_check.cu: the column checks of kv_system_csr (smallest offending entry
// index to *d_first_bad, all ones when none) and the FP32 rounding of values
cudaError_t csr_check_cols_async(const int64_t* d_rp, const int32_t* d_col, int64_t n, unsigned long long* d_first_bad,
                                 cudaStream_t st);
cudaError_t round_to_float_async(const double* src, float* dst, int64_t cnt, cudaStream_t st);
int row_dot_blocks();
int launch_row_dot(Prob* p, int j0, int ncols, void* V, int xslot, int wslot, int it);
int launch_basis_transpose(const Prob* inner, double* out, cudaStream_t st);

// The projection P[:, jcol] = s_jcol C v of a new Krylov vector: done inline
// by the block that finishes the vector for up to PROJ_INLINE_MAX rows of C,
// else by launch_project over the whole grid (one warp per row; the
// transpose dynamics project by E'^T, one row per column of E).
constexpr int PROJ_INLINE_MAX = 16;
int launch_project(Prob* p, int j0, int ncols, const void* w0, int64_t cstride, int jcol);

// generic vectors (k_vector.cu)
int launch_init_norm(Prob* p, int j, void* B);
int launch_scatter(Prob* p, int j, void* B);
int launch_dense_to(Prob* p, int j, void* B);

// CSR (k_csr.cu): Krylov iterations of columns j0 .. j0+ncols-1 (same method),
// whose vector sets start at V (stride nvec * N elements per column)
int launch_csr_columns(Prob* p, int j0, int ncols, void* V, bool lanczos);
int64_t csr_scratch_slots(int64_t N, int m);
int csr_autotune(Prob* p);
size_t csr_xi_bytes(const Prob* p);  // interleaved SpMM input (0 if no candidate uses it)
// per-step LP for polyhedral sets (k_lp.cu)
size_t lp_smem_bytes(int i, int m);
int launch_step_lp(const Prob* p, const double* dU, const double* dv, int qu, const double* dIz,
                   const double* diota, int qi, int m, double* dmargin, int* dstatus, double* dzx, double* dyx,
                   int* dzflag);
size_t csr_arnoldi_dev_bytes();

// exponential + basis (k_expm.cu)
int launch_expm_basis(Prob* p);
// Largest dimension of the shared-memory exponential (k_expm.cu: six m x m
// double matrices per block); above it, and for the PROPAGATE schedule, the
// global-memory exponential (k_expm_large.cu) runs, in batches of
// large_expm_batch runs
constexpr int EXPM_SMEM_M = 64;
size_t large_expm_scratch_doubles(int m, int steps);
int large_expm_batch(int m, int steps, int runs);
int launch_expm_large(Prob* p, int j0, int ncols, int dim, bool write_basis);
inline bool needs_large_expm(int m, int expm_mode) { return m > EXPM_SMEM_M || expm_mode == KV_EXPM_PROPAGATE; }
int expm_prepare(int device);
int fused_prepare();
// one-time set-up that stream capture cannot contain (kv_graph.cu)
int prepare_for_capture(int device);

// bounds (k_bounds.cu)
int launch_bounds(Prob* p);
size_t bounds_scratch_doubles(int ncol, int o, int steps);

// number of reduction partial slots a problem needs
int64_t reduce_slots_needed(const Prob* p);

inline size_t elem_size(int prec) { return prec == KV_FP32 ? 4 : 8; }

}  // namespace kv

// the opaque handles of include/kv.h
struct kv_ctx : public kv::Ctx {};
struct kv_sys : public kv::Sys {};
struct kv_prob : public kv::Prob {};
