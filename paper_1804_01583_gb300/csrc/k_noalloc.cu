// k_noalloc.cu -- grid Lanczos for small grids without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// result: real-time or embedded hosts that reserve all device memory up front
// and forbid allocation afterwards, and callers running inside another
// runtime's allocator or memory-pool callback, which must not re-enter the
// driver's allocator.  For them, kv_grid_lanczos_noalloc runs the projected
// Lanczos iterations on a small grid with every piece of working memory -- the
// two Krylov vectors, the reduction partials, the column state -- in one
// file-scope device array of fixed size.  The caller passes the inputs and the
// output buffers; nothing is allocated or freed, by this file or by any
// library it calls.
//
// The kernels are a variant of the two-pass FP64 grid passes of the main
// path (same arithmetic: alpha_j = v_j . A v_j, then w = A v_j - alpha_j v_j -
// beta_j v_{j-1} stored over v_{j-1}), flattened to one thread per grid point
// in a fixed grid of KV_NA_BLOCKS blocks so the scratch size is known.
//
// C comes as device arrays the host never sees, so the first kernel checks
// them (offsets from 0, never decreasing; column indices inside the grid)
// before anything reads the grid through them; rejected arrays end the call's
// work with m_used = -1.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; calls that overlap on the GPU (on different streams, or
// from different host threads) race on it.  The first call on a device looks
// up the array's device address (cudaGetSymbolAddress) with that device
// current; make that first call before any stream capture begins.  The
// address is kept for the life of the process: after a reset of the device
// (cudaDeviceReset) it is stale, so the entry point must not be called on that
// device again in the same process.
#include <mutex>

#include "kv_internal.h"
#include "reduce.cuh"

namespace kv {

constexpr int NA_NT = 256;
constexpr int NA_BLOCKS = 256;  // fixed grid: partials need NA_BLOCKS slots

struct NaLayout {
    double vec[2][KV_NOALLOC_MAX_N];
    double partials[NA_BLOCKS];
    ColState state;
    unsigned counter;
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NaLayout)];

struct NaGrid {
    int64_t nx, ny, nz, n;
    double kx, ky, kz, kc;
};

__device__ __forceinline__ double na_stencil(const double* B, const NaGrid& g, int64_t i, double* cself) {
    const int64_t x = i % g.nx, y = (i / g.nx) % g.ny, z = i / (g.nx * g.ny);
    const int64_t sy = g.nx, sz = g.nx * g.ny;
    const double c = B[i];
    const double l = x > 0 ? B[i - 1] : 0.0, r = x < g.nx - 1 ? B[i + 1] : 0.0;
    const double d = y > 0 ? B[i - sy] : 0.0, u = y < g.ny - 1 ? B[i + sy] : 0.0;
    const double b = z > 0 ? B[i - sz] : 0.0, f = z < g.nz - 1 ? B[i + sz] : 0.0;
    *cself = c;
    return g.kx * (l + r) + g.ky * (d + u) + g.kz * (b + f);  // the centre term is added by the caller
}

// Whether C's CSR arrays stay inside the grid of n points: the offsets start
// at 0 and never decrease, and every column index lies in [0, n).  Run by all
// threads of one block; only entries inside the given offsets are read.
__device__ bool na_check_C(const CDesc& cd, int64_t n, int* bad) {
    if (threadIdx.x == 0) *bad = (cd.o > 0 && cd.rp[0] != 0) ? 1 : 0;
    __syncthreads();
    for (int r = threadIdx.x; r < cd.o; r += NA_NT)
        if (cd.rp[r + 1] < cd.rp[r]) *bad = 1;
    __syncthreads();
    if (!*bad && cd.o > 0) {
        for (int64_t e = threadIdx.x; e < cd.rp[cd.o]; e += NA_NT) {
            const int64_t c = cd.col[e];
            if (c < 0 || c >= n) *bad = 1;
        }
    }
    __syncthreads();
    return *bad == 0;
}

// P[:, col] = scale * C x; entries whose column lies outside the grid are
// skipped (the first kernel has rejected such arrays already)
__device__ void na_gather_P(const CDesc& cd, const double* x, int64_t n, double scale, double* P, int m, int col,
                            double* sh) {
    for (int r = 0; r < cd.o; ++r) {
        double v = 0.0;
        for (int64_t e = cd.rp[r] + threadIdx.x; e < cd.rp[r + 1]; e += NA_NT) {
            const int64_t c = cd.col[e];
            if (c >= 0 && c < n) v += cd.val[e] * __ldcg(x + c);
        }
        v = block_sum<NA_NT>(v, sh);
        if (threadIdx.x == 0) P[(int64_t)r * m + col] = scale * v;
    }
}

__global__ void __launch_bounds__(NA_NT) k_na_init(NaLayout* L, NaGrid g, int64_t lx, int64_t ly, int64_t lz,
                                                   int64_t hx, int64_t hy, int64_t hz, double value, CDesc cd,
                                                   int m, double* P, double* beta0_out, int* m_used_out) {
    __shared__ double sh[NA_NT / 32];
    __shared__ int flag;
    double* B = L->vec[0];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * NA_NT + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * NA_NT) {
        const int64_t x = i % g.nx, y = (i / g.nx) % g.ny, z = i / (g.nx * g.ny);
        const bool in = x >= lx && x < hx && y >= ly && y < hy && z >= lz && z < hz;
        B[i] = in ? value : 0.0;
        if (in) acc = fma(value, value, acc);
    }
    const double part = block_sum<NA_NT>(acc, sh);
    if (!grid_arrive(part, L->partials, &L->counter, blockIdx.x, gridDim.x, &flag)) return;
    const double tot = grid_finish<NA_NT>(L->partials, gridDim.x, &L->counter, sh);
    __shared__ double s0;
    __shared__ int c_bad;
    const bool c_ok = na_check_C(cd, g.n, &c_bad);
    if (threadIdx.x == 0) {
        const double b0 = sqrt(tot);
        ColState* st = &L->state;
        st->beta0 = b0;
        st->status = 0;
        st->m_used = m;
        *beta0_out = b0;
        if (!(b0 > 0.0) || !isfinite(b0)) {
            st->done = 1;
            st->m_used = 0;
            s0 = 0.0;
        } else {
            st->done = 0;
            st->s[0] = 1.0 / b0;
            s0 = 1.0 / b0;
        }
        if (!c_ok) {  // nothing runs: the later kernels see done
            st->done = 1;
            st->m_used = -1;
            st->status |= 2;
        }
        *m_used_out = st->m_used;
    }
    __syncthreads();
    if (!c_ok) return;
    na_gather_P(cd, B, g.n, s0, P, m, 0, sh);
}

__global__ void __launch_bounds__(NA_NT) k_na_alpha(NaLayout* L, NaGrid g, int j, double* H, int m) {
    ColState* st = &L->state;
    if (st->done) return;
    __shared__ double sh[NA_NT / 32];
    __shared__ int flag;
    const double* B = L->vec[j & 1];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * NA_NT + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * NA_NT) {
        double c;
        const double nb = na_stencil(B, g, i, &c);
        acc = fma(c, nb + g.kc * c, acc);
    }
    const double part = block_sum<NA_NT>(acc, sh);
    if (!grid_arrive(part, L->partials, &L->counter, blockIdx.x, gridDim.x, &flag)) return;
    const double tot = grid_finish<NA_NT>(L->partials, gridDim.x, &L->counter, sh);
    if (threadIdx.x == 0) H[(int64_t)j * m + j] = st->s[j] * st->s[j] * tot;
}

__global__ void __launch_bounds__(NA_NT) k_na_update(NaLayout* L, NaGrid g, int j, double* H, double* P, CDesc cd,
                                                     int m, int* m_used_out) {
    ColState* st = &L->state;
    if (st->done) return;
    __shared__ double sh[NA_NT / 32];
    __shared__ int flag;
    const double* B = L->vec[j & 1];
    double* A = L->vec[(j + 1) & 1];
    const double sj = st->s[j];
    const double alpha = H[(int64_t)j * m + j];
    const double c2 = sj * (g.kc - alpha);
    const double c3 = j == 0 ? 0.0 : -H[(int64_t)j * m + (j - 1)] * st->s[j - 1];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * NA_NT + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * NA_NT) {
        double c;
        const double nb = na_stencil(B, g, i, &c);
        double w = sj * nb + c2 * c;
        if (j > 0) w += c3 * A[i];
        A[i] = w;
        acc = fma(w, w, acc);
    }
    const double part = block_sum<NA_NT>(acc, sh);
    if (!grid_arrive(part, L->partials, &L->counter, blockIdx.x, gridDim.x, &flag)) return;
    const double tot = grid_finish<NA_NT>(L->partials, gridDim.x, &L->counter, sh);
    __shared__ double snext;
    __shared__ int cont;
    if (threadIdx.x == 0) {
        const double beta = sqrt(tot);
        H[(int64_t)(j + 1) * m + j] = beta;
        const double bj = j == 0 ? 0.0 : H[(int64_t)j * m + (j - 1)];
        const double nav = sqrt(alpha * alpha + bj * bj + beta * beta);
        if (!(beta > 1e-12 * nav) || !isfinite(beta)) {
            st->done = 1;
            st->m_used = j + 1;
            *m_used_out = j + 1;
            cont = 0;
        } else {
            if (j + 1 < m) H[(int64_t)j * m + (j + 1)] = beta;
            st->s[j + 1] = 1.0 / beta;
            snext = 1.0 / beta;
            cont = j + 1 < m ? 1 : 0;
        }
    }
    __syncthreads();
    if (cont) na_gather_P(cd, A, g.n, snext, P, m, j + 1, sh);
}

// device address of the scratch array, looked up once per device
static std::mutex g_na_mutex;
static void* g_na_ptr[64] = {nullptr};

static int na_setup(int device, NaLayout** out) {
    if (device < 0 || device >= 64) {
        set_error("kv_grid_lanczos_noalloc: device %d out of range", device);
        return KV_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("kv_grid_lanczos_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return KV_ECUDA;
        }
        g_na_ptr[device] = p;
    }
    *out = (NaLayout*)g_na_ptr[device];
    return KV_OK;
}

}  // namespace kv

extern "C" int kv_grid_lanczos_noalloc(int device, void* stream, int ndim, const int64_t dims[3], double coef,
                                       const double h[3], const int64_t box_lo[3], const int64_t box_hi[3],
                                       double value, int32_t o, const int64_t* c_row_ptr, const int64_t* c_col,
                                       const double* c_val, int32_t krylov_m, double* H, double* P, double* beta0,
                                       int32_t* m_used) {
    using namespace kv;
    if (!dims || !h || !box_lo || !box_hi || !H || !P || !beta0 || !m_used ||
        (o > 0 && (!c_row_ptr || !c_col || !c_val))) {
        set_error("kv_grid_lanczos_noalloc: NULL argument");
        return KV_EINVAL;
    }
    if (ndim != 2 && ndim != 3) {
        set_error("kv_grid_lanczos_noalloc: ndim must be 2 or 3");
        return KV_EINVAL;
    }
    NaGrid g;
    g.nx = dims[0];
    g.ny = dims[1];
    g.nz = ndim == 3 ? dims[2] : 1;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) {
        set_error("kv_grid_lanczos_noalloc: dims must be >= 1");
        return KV_EINVAL;
    }
    if (g.nx > KV_NOALLOC_MAX_N || g.ny > KV_NOALLOC_MAX_N || g.nz > KV_NOALLOC_MAX_N ||
        g.nx * g.ny * g.nz > (int64_t)KV_NOALLOC_MAX_N) {
        set_error("kv_grid_lanczos_noalloc: grid of %lld x %lld x %lld points exceeds the fixed scratch "
                  "(KV_NOALLOC_MAX_N = %d points); use kv_problem/kv_run for larger grids",
                  (long long)g.nx, (long long)g.ny, (long long)g.nz, KV_NOALLOC_MAX_N);
        return KV_EINVAL;
    }
    if (krylov_m < 1 || krylov_m > KV_MAX_M || o < 0) {
        set_error("kv_grid_lanczos_noalloc: krylov_m must be in [1, %d] and o >= 0", KV_MAX_M);
        return KV_EINVAL;
    }
    for (int a = 0; a < ndim; ++a) {
        if (!(h[a] > 0) || box_lo[a] < 0 || box_hi[a] > dims[a] || box_lo[a] > box_hi[a]) {
            set_error("kv_grid_lanczos_noalloc: h or box out of range on axis %d", a);
            return KV_EINVAL;
        }
    }
    g.n = g.nx * g.ny * g.nz;
    g.kx = coef / (h[0] * h[0]);
    g.ky = coef / (h[1] * h[1]);
    g.kz = ndim == 3 ? coef / (h[2] * h[2]) : 0.0;
    g.kc = -2.0 * (g.kx + g.ky + g.kz);
    // the caller's current device is made current again on return
    DeviceGuard dg(device);
    cudaError_t e = dg.err;
    if (e != cudaSuccess) {
        set_error("kv_grid_lanczos_noalloc: cudaSetDevice: %s", cudaGetErrorString(e));
        return KV_ECUDA;
    }
    NaLayout* L = nullptr;
    int rc = na_setup(device, &L);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int m = krylov_m;
    // what must start at zero: the reduction ticket and the output matrices
    e = cudaMemsetAsync(&L->counter, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(H, 0, sizeof(double) * (size_t)(m + 1) * m, s);
    if (e == cudaSuccess && o > 0) e = cudaMemsetAsync(P, 0, sizeof(double) * (size_t)o * m, s);
    if (e != cudaSuccess) {
        set_error("kv_grid_lanczos_noalloc: cudaMemsetAsync: %s", cudaGetErrorString(e));
        return KV_ECUDA;
    }
    const int64_t lz = ndim == 3 ? box_lo[2] : 0, hz = ndim == 3 ? box_hi[2] : 1;
    CDesc cd{o, c_row_ptr, c_col, c_val, g.n};
    k_na_init<<<NA_BLOCKS, NA_NT, 0, s>>>(L, g, box_lo[0], box_lo[1], lz, box_hi[0], box_hi[1], hz, value, cd, m, P,
                                          beta0, m_used);
    for (int j = 0; j < m; ++j) {
        k_na_alpha<<<NA_BLOCKS, NA_NT, 0, s>>>(L, g, j, H, m);
        k_na_update<<<NA_BLOCKS, NA_NT, 0, s>>>(L, g, j, H, P, cd, m, m_used);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kv_grid_lanczos_noalloc: launch failed: %s", cudaGetErrorString(e));
        return KV_ECUDA;
    }
    return KV_OK;
}
