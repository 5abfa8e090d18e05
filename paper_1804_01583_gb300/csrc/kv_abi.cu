// kv_abi.cu -- the C ABI of include/kv.h: contexts, the device-memory arena,
// systems, problems and the enqueue of the whole path on one stream.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "kv_internal.h"

namespace kv {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

static int fail(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// ------------------------------------------------------------------- arena
static const size_t kAlign = 256;

void Arena::init(char* base, size_t size) {
    base_ = base;
    size_ = size;
    in_use_ = 0;
    free_.clear();
    used_.clear();
    if (size) free_[0] = size;
}

void* Arena::alloc(size_t bytes) {
    if (bytes == 0) bytes = 1;
    if (bytes > size_) return nullptr;  // also keeps the rounding below from wrapping
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second >= bytes) {
            const size_t off = it->first, sz = it->second;
            free_.erase(it);
            if (sz > bytes) free_[off + bytes] = sz - bytes;
            used_[off] = bytes;
            in_use_ += bytes;
            return base_ + off;
        }
    }
    return nullptr;
}

void Arena::free(void* p) {
    if (!p) return;
    const size_t off = (size_t)((char*)p - base_);
    auto it = used_.find(off);
    if (it == used_.end()) return;
    size_t sz = it->second;
    used_.erase(it);
    in_use_ -= sz;
    size_t start = off;
    auto nx = free_.lower_bound(off);
    if (nx != free_.end() && nx->first == off + sz) {
        sz += nx->second;
        free_.erase(nx);
    }
    auto pv = free_.lower_bound(off);
    if (pv != free_.begin()) {
        --pv;
        if (pv->first + pv->second == off) {
            start = pv->first;
            sz += pv->second;
            free_.erase(pv);
        }
    }
    free_[start] = sz;
}

size_t Arena::largest_free() const {
    size_t b = 0;
    for (auto& kv : free_) b = std::max(b, kv.second);
    return b;
}

// ----------------------------------------------------------- launch scope
bool dep_launch_ok(const Ctx* c) {
    static const bool env_on = [] {
        const char* e = getenv("KV_PDL");
        return !(e && e[0] == '0');
    }();
    return env_on && !c->profiling && !c->capturing;
}

LaunchScope::LaunchScope(Ctx* c, const char* name) : ctx(c) {
    ctx->launches++;
    if (!ctx->profiling) return;
    Ctx::Rec r;
    r.name = name;
    for (int q = 0; q < 2; ++q) {
        cudaEvent_t e;
        if (!ctx->spare_events.empty()) {
            e = ctx->spare_events.back();
            ctx->spare_events.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            return;
        }
        (q == 0 ? r.a : r.b) = e;
    }
    cudaEventRecord(r.a, ctx->stream);
    ctx->recs.push_back(r);
    rec = (int)ctx->recs.size() - 1;
}

LaunchScope::~LaunchScope() {
    if (rec >= 0) cudaEventRecord(ctx->recs[rec].b, ctx->stream);
}

static void clear_profile(Ctx* c) {
    for (auto& r : c->recs) {
        c->spare_events.push_back(r.a);
        c->spare_events.push_back(r.b);
    }
    c->recs.clear();
}

// ------------------------------------------------------------- helpers
template <typename T>
static int dalloc(Prob* p, T** out, size_t count) {
    if (count > SIZE_MAX / sizeof(T)) return fail(KV_ENOMEM, "device allocation size overflows");
    void* q = p->ctx->arena.alloc(count * sizeof(T));
    if (!q) {
        return fail(KV_ENOMEM, "device pool exhausted: need %zu more bytes (largest free block %zu of %zu)",
                    count * sizeof(T), p->ctx->arena.largest_free(), p->ctx->arena.total());
    }
    p->allocs.push_back(q);
    *out = (T*)q;
    return KV_OK;
}

static int upload(Ctx* c, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return KV_OK;
    KV_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return KV_OK;
}

int64_t reduce_slots_needed(const Prob* p) {
    int64_t nb = 152 * 8;
    if (p->sys->kind == 0) {
        StencilGeom g;
        g.nx = p->sys->dims[0];
        g.ny = p->sys->ndim >= 2 ? p->sys->dims[1] : 1;
        g.nz = p->sys->ndim >= 3 ? p->sys->dims[2] : 1;
        int zc;
        nb = std::max<int64_t>(nb, stencil_blocks(g, &zc));
        if (p->fused) nb = std::max<int64_t>(nb, 2 * (int64_t)fused_tma_blocks(p, &zc));
        if (p->fused64) nb = std::max<int64_t>(nb, 2 * (int64_t)fused64_blocks(p));
        return nb * (int64_t)(p->m + 2);
    }
    // CSR: one region of partials per column (all columns run together)
    return std::max<int64_t>(nb, (int64_t)p->i * csr_scratch_slots(p->N, p->m));
}

// Vector sets: grid problems run their columns one after another on one set;
// CSR problems run all columns of a method together, one set per column.
static int vector_sets(const Sys* s, int i) { return s->kind == 0 ? 1 : i; }

}  // namespace kv

using namespace kv;

extern "C" {

const char* kv_version(void) { return "kv 0.1 (sm_103a)"; }

const char* kv_last_error(void) { return g_err.c_str(); }

int kv_create(kv_ctx** out, int device, void* pool, size_t pool_bytes, void* stream) {
    if (!out) return fail(KV_EINVAL, "kv_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    KV_CHECK_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(KV_EINVAL, "kv_create: device %d of %d", device, ndev);
    if (pool && ((uintptr_t)pool % 256) != 0) return fail(KV_EINVAL, "kv_create: pool must be 256-byte aligned");
    if (pool_bytes < 4096) return fail(KV_EINVAL, "kv_create: pool_bytes too small");
    KV_WITH_DEVICE(device);
    int rc = KV_OK;
    kv_ctx* c = new (std::nothrow) kv_ctx();
    if (!c) return fail(KV_ENOMEM, "kv_create: host allocation");
    c->device = device;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(KV_ECUDA, "kv_create: cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    if (pool) {
        c->pool = pool;
    } else {
        cudaError_t e = cudaMalloc(&c->pool, pool_bytes);
        if (e != cudaSuccess) {
            if (c->own_stream) cudaStreamDestroy(c->stream);
            delete c;
            return fail(KV_ENOMEM, "kv_create: cudaMalloc(%zu) failed: %s", pool_bytes, cudaGetErrorString(e));
        }
        c->own_pool = true;
    }
    c->arena.init((char*)c->pool, pool_bytes);
    *out = c;
    return KV_OK;
}

int kv_destroy(kv_ctx* c) {
    if (!c) return KV_OK;
    ::kv::DeviceGuard kv_device_guard_(c->device);
    cudaStreamSynchronize(c->stream);
    clear_profile(c);
    for (auto e : c->spare_events) cudaEventDestroy(e);
    if (c->own_pool) cudaFree(c->pool);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return KV_OK;
}

int kv_pool_stats(const kv_ctx* c, size_t* in_use, size_t* total) {
    if (!c) return fail(KV_EINVAL, "kv_pool_stats: ctx is NULL");
    if (in_use) *in_use = c->arena.in_use();
    if (total) *total = c->arena.total();
    return KV_OK;
}

int kv_launch_count(const kv_ctx* c, int64_t* launches) {
    if (!c || !launches) return fail(KV_EINVAL, "kv_launch_count: NULL argument");
    *launches = c->launches;
    return KV_OK;
}

int kv_system_stencil(kv_ctx* c, kv_sys** out, int ndim, const int64_t dims[3], double coef, const double h[3],
                      const double* b) {
    return kv_system_grid(c, out, ndim, dims, coef, h, nullptr, b);
}

int kv_system_grid(kv_ctx* c, kv_sys** out, int ndim, const int64_t dims[3], double coef, const double h[3],
                   const double* face, const double* b) {
    if (!c || !out || !dims || !h) return fail(KV_EINVAL, "kv_system_stencil: NULL argument");
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return fail(KV_EINVAL, "kv_system_stencil: ndim must be 2 or 3");
    int64_t n = 1;
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 1 || dims[a] > (int64_t)1 << 31) return fail(KV_EINVAL, "kv_system_stencil: dims[%d]", a);
        if (!(h[a] > 0) || !isfinite(h[a])) return fail(KV_EINVAL, "kv_system_stencil: h[%d]", a);
        if (n > ((int64_t)1 << 62) / dims[a]) return fail(KV_EINVAL, "kv_system_stencil: grid too large");
        n *= dims[a];
    }
    if (!isfinite(coef)) return fail(KV_EINVAL, "kv_system_stencil: coef");
    if (face) {
        for (int f = 0; f < 2 * ndim; ++f)
            if (!isfinite(face[f]) || face[f] < 0.0)
                return fail(KV_EINVAL, "kv_system_grid: face[%d] must be finite and >= 0", f);
        // the grid kernels hold a face as its share gamma / kappa of the
        // coupling it replaces, which needs kappa > 0
        if (!(coef > 0.0)) return fail(KV_EINVAL, "kv_system_grid: face coefficients need coef > 0");
    }
    // launch-shape limits of the grid kernels: ceil(ny/8) and ceil(nz/8) blocks
    if (dims[1] > 524280 || (ndim == 3 && dims[2] > 524280))
        return fail(KV_EINVAL, "kv_system_stencil: ny and nz must be <= 524280");
    KV_WITH_DEVICE(c->device);
    int rc = KV_OK;
    kv_sys* s = new (std::nothrow) kv_sys();
    if (!s) return fail(KV_ENOMEM, "host allocation");
    s->ctx = c;
    s->kind = 0;
    s->ndim = ndim;
    for (int a = 0; a < 3; ++a) {
        s->dims[a] = a < ndim ? dims[a] : 1;
        s->h[a] = a < ndim ? h[a] : 1.0;
    }
    s->coef = coef;
    s->n = n;
    s->symmetric = true;
    // the boundary: gamma per face, Dirichlet-0 (gamma = coef / h_a^2) unless given
    s->faces = false;
    for (int a = 0; a < ndim; ++a) {
        const double kap = coef / (s->h[a] * s->h[a]);
        for (int side = 0; side < 2; ++side) {
            s->face[2 * a + side] = face ? face[2 * a + side] : kap;
            if (s->face[2 * a + side] != kap) s->faces = true;
        }
    }
    s->mu = 0.0;
    if (!s->faces) {
        // largest eigenvalue of the Dirichlet-0 Laplacian: the Kronecker sum of the
        // 1-D second differences' largest eigenvalues -(4/h^2) sin^2(pi / (2(N+1)))
        for (int a = 0; a < ndim; ++a) {
            const double sn = sin(M_PI / (2.0 * (double)(s->dims[a] + 1)));
            s->mu -= coef * 4.0 / (s->h[a] * s->h[a]) * sn * sn;
        }
    } else {
        // Gershgorin bound of the (symmetric) operator: a point's diagonal is
        // -sum over its neighbours of kappa - sum over its faces of gamma, its
        // off-diagonal sum that of |kappa|; with gamma >= 0 the largest row
        // value is at most 2 sum_a (|kappa_a| - kappa_a) (0 for coef >= 0)
        for (int a = 0; a < ndim; ++a) {
            const double kap = coef / (s->h[a] * s->h[a]);
            s->mu += 2.0 * (fabs(kap) - kap);
        }
    }
    s->mu_aug = s->mu;
    if (!b) {  // Gershgorin: |diagonal| + off-diagonal sum <= 4 sum_a |kappa_a| + sum_f gamma_f
        double nb = 0.0;
        for (int a = 0; a < ndim; ++a) nb += 4.0 * fabs(coef / (s->h[a] * s->h[a]));
        for (int f = 0; f < 6; ++f) nb += s->face[f];
        s->norm2_bound = nb * (1.0 + 1e-12);
    }
    if (b) {
        s->d_b = (double*)c->arena.alloc((size_t)n * sizeof(double));
        if (!s->d_b) {
            delete s;
            return fail(KV_ENOMEM, "kv_system_stencil: pool cannot hold b");
        }
        rc = upload(c, s->d_b, b, (size_t)n * sizeof(double));
        if (rc) {
            c->arena.free(s->d_b);
            delete s;
            return rc;
        }
    }
    *out = s;
    return KV_OK;
}

int kv_system_csr(kv_ctx* c, kv_sys** out, int64_t n, const int64_t* row_ptr, const int32_t* col,
                  const double* val, const double* b, int symmetric, int value_precision, int on_device) {
    if (!c || !out || !row_ptr || !col || !val) return fail(KV_EINVAL, "kv_system_csr: NULL argument");
    *out = nullptr;
    if (n < 1 || n >= ((int64_t)1 << 31)) return fail(KV_EINVAL, "kv_system_csr: n out of range");
    if (value_precision != KV_FP64 && value_precision != KV_FP32)
        return fail(KV_EINVAL, "kv_system_csr: value_precision");
    KV_WITH_DEVICE(c->device);
    int rc = KV_OK;
    // the row pointers bound every read of the other arrays and size the
    // allocations: checked on the host (device arrays: one copy to the host)
    std::vector<int64_t> hrp;
    const int64_t* rp = row_ptr;
    if (on_device) {
        hrp.resize((size_t)n + 1);
        KV_CHECK_CUDA(cudaMemcpy(hrp.data(), row_ptr, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        rp = hrp.data();
    }
    if (rp[0] != 0) return fail(KV_EINVAL, "kv_system_csr: row_ptr[0] != 0");
    for (int64_t r = 0; r < n; ++r)
        if (rp[r + 1] < rp[r]) return fail(KV_EINVAL, "kv_system_csr: row_ptr decreases at row %lld", (long long)r);
    const int64_t nnz = rp[n];
    kv_sys* s = new (std::nothrow) kv_sys();
    if (!s) return fail(KV_ENOMEM, "host allocation");
    s->ctx = c;
    s->kind = 1;
    s->n = n;
    s->nnz = nnz;
    s->symmetric = symmetric != 0;
    s->val_prec = value_precision;
    const size_t vb = (size_t)nnz * elem_size(value_precision);
    s->d_rp = (int64_t*)c->arena.alloc((size_t)(n + 1) * sizeof(int64_t));
    s->d_col = (int32_t*)c->arena.alloc((size_t)std::max<int64_t>(nnz, 1) * sizeof(int32_t));
    s->d_val = c->arena.alloc(std::max<size_t>(vb, 8));
    if (b) s->d_b = (double*)c->arena.alloc((size_t)n * sizeof(double));
    unsigned long long* d_bad = (unsigned long long*)c->arena.alloc(sizeof(unsigned long long));
    auto release = [&]() {
        c->arena.free(s->d_rp);
        c->arena.free(s->d_col);
        c->arena.free(s->d_val);
        c->arena.free(s->d_b);
        c->arena.free(d_bad);
        delete s;
    };
    if (!s->d_rp || !s->d_col || !s->d_val || (b && !s->d_b) || !d_bad) {
        release();
        return fail(KV_ENOMEM, "kv_system_csr: pool cannot hold the matrix (%lld nnz)", (long long)nnz);
    }
    // FP32 values from doubles: a staging buffer for host doubles, the largest
    // of a few sizes the pool holds
    double* stage = nullptr;
    int64_t stage_n = 0;
    if (value_precision == KV_FP32 && !on_device && nnz > 0) {
        for (int64_t want : {(int64_t)1 << 22, (int64_t)1 << 19, (int64_t)1 << 16}) {
            stage_n = std::min<int64_t>(want, nnz);
            stage = (double*)c->arena.alloc((size_t)stage_n * sizeof(double));
            if (stage) break;
        }
        if (!stage) {
            release();
            return fail(KV_ENOMEM, "kv_system_csr: pool cannot hold the value staging buffer");
        }
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaStream_t st = c->stream;
    cudaError_t e = cudaMemcpyAsync(s->d_rp, row_ptr, (size_t)(n + 1) * sizeof(int64_t), kind, st);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(s->d_col, col, (size_t)nnz * sizeof(int32_t), kind, st);
    if (e == cudaSuccess) e = csr_check_cols_async(s->d_rp, s->d_col, n, d_bad, st);
    if (e == cudaSuccess && nnz > 0) {
        if (value_precision == KV_FP64) {
            e = cudaMemcpyAsync(s->d_val, val, (size_t)nnz * sizeof(double), kind, st);
        } else if (on_device) {
            e = round_to_float_async(val, (float*)s->d_val, nnz, st);
        } else {
            for (int64_t q = 0; q < nnz && e == cudaSuccess; q += stage_n) {
                const int64_t cnt = std::min<int64_t>(stage_n, nnz - q);
                e = cudaMemcpyAsync(stage, val + q, (size_t)cnt * sizeof(double), cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess) e = round_to_float_async(stage, (float*)s->d_val + q, cnt, st);
            }
        }
    }
    if (e == cudaSuccess && b) e = cudaMemcpyAsync(s->d_b, b, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
    unsigned long long first_bad = ~0ULL;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&first_bad, d_bad, sizeof(first_bad), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    c->arena.free(stage);
    if (e != cudaSuccess) {
        release();
        return fail(KV_ECUDA, "kv_system_csr: upload failed: %s", cudaGetErrorString(e));
    }
    if (first_bad != ~0ULL) {  // the first offending entry in storage order
        const int64_t at = (int64_t)first_bad;
        const int64_t r = (int64_t)(std::upper_bound(rp, rp + n + 1, at) - rp) - 1;
        int32_t v = 0;
        if (on_device)
            e = cudaMemcpy(&v, col + at, sizeof(v), cudaMemcpyDeviceToHost);
        else
            v = col[at];
        release();
        if (e != cudaSuccess) return fail(KV_ECUDA, "kv_system_csr: %s", cudaGetErrorString(e));
        if (v < 0 || (int64_t)v >= n)
            return fail(KV_EINVAL, "kv_system_csr: col[%lld] = %d out of range", (long long)at, v);
        return fail(KV_EINVAL, "kv_system_csr: row %lld columns not strictly increasing", (long long)r);
    }
    c->arena.free(d_bad);
    d_bad = nullptr;
    double rmax = INFINITY;
    rc = csr_lognorm_bounds(s, b, &s->mu, &s->mu_aug, &rmax);
    if (!rc && s->symmetric && !b) s->norm2_bound = rmax;  // ||A||_2 <= ||A||_inf for symmetric A
    if (rc) {
        release();
        return rc;
    }
    *out = s;
    return KV_OK;
}

int kv_sys_destroy(kv_sys* s) {
    if (!s) return KV_OK;
    Ctx* c = s->ctx;
    ::kv::DeviceGuard kv_device_guard_(c->device);
    cudaStreamSynchronize(c->stream);
    c->arena.free(s->d_rp);
    c->arena.free(s->d_col);
    c->arena.free(s->d_val);
    c->arena.free(s->d_b);
    c->arena.free(s->d_rpT);
    c->arena.free(s->d_colT);
    c->arena.free(s->d_valT);
    delete s;
    return KV_OK;
}

// ---------------------------------------------------------------- problems
// KV_PREC_AUTO: FP64 storage when the operator is symmetric and its largest
// eigenvalue bound mu gives mu T > -1 over the horizon T = steps dt (its
// slowest mode loses less than a factor e, so the rounding of FP32-stored
// Krylov vectors in that mode reaches the last outputs undamped), else FP32.
// A CSR system keeps the value precision it was created with: when the rule
// asks for FP64 and the values are FP32 the problem is refused.
static int resolve_precision(const Sys* s, const kv_problem_desc* d, int precision, int* out) {
    *out = precision;
    if (precision != KV_PREC_AUTO) return KV_OK;
    const double T = d ? (double)d->steps * d->dt : 0.0;
    const bool conserving = s->symmetric && s->mu * T > -1.0;
    *out = conserving ? KV_FP64 : KV_FP32;
    if (s->kind == 1) {
        if (conserving && s->val_prec != KV_FP64)
            return fail(KV_EINVAL, "KV_PREC_AUTO: the operator keeps a slow mode over the horizon (mu T = %g > -1), "
                        "so FP32 storage does not meet its accuracy; create the CSR system with KV_FP64 values",
                        s->mu * T);
        *out = s->val_prec;
    }
    return KV_OK;
}

static int validate(const Sys* s, const kv_problem_desc* d, int precision) {
    if (!d) return fail(KV_EINVAL, "problem description is NULL");
    if (precision != KV_FP64 && precision != KV_FP32) return fail(KV_EINVAL, "precision");
    if (s->kind == 1 && s->val_prec != precision)
        return fail(KV_EINVAL, "problem precision must match the CSR value precision");
    if (d->i < 1 || !d->cols) return fail(KV_EINVAL, "need at least one column");
    if (d->o < 1 || !d->c_row_ptr || !d->theta) return fail(KV_EINVAL, "need at least one output row");
    if (!(d->dt > 0) || !isfinite(d->dt)) return fail(KV_EINVAL, "dt must be positive and finite");
    if (d->steps < 0) return fail(KV_EINVAL, "steps must be >= 0");
    bool any_arnoldi = false;
    for (int j = 0; d->cols && j < d->i; ++j) {
        const bool carries = s->d_b != nullptr && d->cols[j].is_fixed;
        any_arnoldi = any_arnoldi || d->method == KV_ARNOLDI ||
                      (d->method == KV_AUTO && !(s->symmetric && !carries));
    }
    const int mmax = any_arnoldi ? KV_MAX_M : KV_MAX_M_LANCZOS;
    if (d->krylov_m < 1 || d->krylov_m > mmax)
        return fail(KV_EINVAL, "krylov_m must be in [1, %d]%s", mmax, any_arnoldi ? " (Arnoldi columns)" : "");
    if ((int64_t)(d->steps + 1) * d->o >= ((int64_t)1 << 31) - 1) return fail(KV_EINVAL, "o * (steps+1) too large");
    if (d->method < KV_AUTO || d->method > KV_ARNOLDI) return fail(KV_EINVAL, "method");
    if (d->expm_mode != KV_EXPM_PER_STEP && d->expm_mode != KV_EXPM_PROPAGATE) return fail(KV_EINVAL, "expm_mode");
    if (isnan(d->err_target)) return fail(KV_EINVAL, "err_target is NaN");
    if (d->simulate < KV_SIM_FORWARD || d->simulate > KV_SIM_AUTO) return fail(KV_EINVAL, "simulate");
    const int64_t n = s->n;
    if (d->c_row_ptr[0] != 0) return fail(KV_EINVAL, "c_row_ptr[0] != 0");
    for (int r = 0; r < d->o; ++r) {
        if (d->c_row_ptr[r + 1] < d->c_row_ptr[r]) return fail(KV_EINVAL, "c_row_ptr decreases");
        if (isnan(d->theta[r])) return fail(KV_EINVAL, "theta[%d] is NaN", r);
    }
    const int64_t cnnz = d->c_row_ptr[d->o];
    if (cnnz > 0 && (!d->c_col || !d->c_val)) return fail(KV_EINVAL, "C arrays are NULL");
    for (int64_t e = 0; e < cnnz; ++e) {
        if (d->c_col[e] < 0 || d->c_col[e] >= n) return fail(KV_EINVAL, "c_col[%lld] out of range", (long long)e);
        if (!isfinite(d->c_val[e])) return fail(KV_EINVAL, "c_val[%lld] not finite", (long long)e);
    }
    for (int j = 0; j < d->i; ++j) {
        const kv_column& c = d->cols[j];
        if (!(c.zlo <= c.zhi) || !isfinite(c.zlo) || !isfinite(c.zhi)) return fail(KV_EINVAL, "column %d: zlo > zhi", j);
        if (c.is_fixed && (c.zlo != 1.0 || c.zhi != 1.0)) return fail(KV_EINVAL, "column %d: fixed needs z = 1", j);
        if (c.kind == KV_COL_BOX) {
            if (s->kind != 0) return fail(KV_EINVAL, "column %d: box columns need a grid system", j);
            for (int a = 0; a < s->ndim; ++a)
                if (c.box_lo[a] < 0 || c.box_hi[a] > s->dims[a] || c.box_lo[a] > c.box_hi[a])
                    return fail(KV_EINVAL, "column %d: box out of the grid on axis %d", j, a);
            if (!isfinite(c.value)) return fail(KV_EINVAL, "column %d: value", j);
        } else if (c.kind == KV_COL_SPARSE) {
            if (c.nnz < 0 || (c.nnz > 0 && (!c.idx || !c.val))) return fail(KV_EINVAL, "column %d: sparse arrays", j);
            std::vector<int64_t> ix(c.idx, c.idx + c.nnz);
            std::sort(ix.begin(), ix.end());
            for (int64_t e = 0; e < c.nnz; ++e) {
                if (ix[e] < 0 || ix[e] >= n) return fail(KV_EINVAL, "column %d: index out of range", j);
                if (e > 0 && ix[e] == ix[e - 1]) return fail(KV_EINVAL, "column %d: duplicate index", j);
                if (!isfinite(c.val[e])) return fail(KV_EINVAL, "column %d: value not finite", j);
            }
        } else if (c.kind == KV_COL_DENSE) {
            if (!c.dense) return fail(KV_EINVAL, "column %d: dense is NULL", j);
        } else {
            return fail(KV_EINVAL, "column %d: kind", j);
        }
        const bool carries = s->d_b != nullptr && c.is_fixed;
        if (carries && s->kind == 0) return fail(KV_EINVAL, "column %d: forcing term on grid systems is not supported", j);
        if (d->method == KV_LANCZOS && (carries || !s->symmetric))
            return fail(KV_EINVAL, "column %d: Lanczos needs a symmetric operator", j);
        if (s->kind == 0 && d->method == KV_ARNOLDI)
            return fail(KV_EINVAL, "Arnoldi on grid systems is not supported; grids are symmetric (use Lanczos)");
    }
    return KV_OK;
}

// How a problem is built: the default, or the inner problem of the
// transpose dynamics (its runs start at the rows of C with constant entry 0;
// with trans_aug they run on A'^T, whose last row is b . x).
struct BuildOpts {
    bool trans_runs = false;
    int trans_aug = 0;
    const double* brow = nullptr;
};

static void plan_methods(const Sys* s, const kv_problem_desc* d, Prob* p, const BuildOpts& bo = BuildOpts{}) {
    p->method.resize(d->i);
    p->aug.resize(d->i);
    for (int j = 0; j < d->i; ++j) {
        const bool carries = bo.trans_runs ? bo.trans_aug != 0 : (s->d_b != nullptr && d->cols[j].is_fixed != 0);
        p->aug[j] = carries ? 1 : 0;
        int m = d->method;
        if (m == KV_AUTO) m = (s->symmetric && !carries) ? KV_LANCZOS : KV_ARNOLDI;
        p->method[j] = m;
    }
}

static bool runs_transposed(const kv_problem_desc* d) {
    return d->simulate == KV_SIM_TRANSPOSE || (d->simulate == KV_SIM_AUTO && d->o < d->i);
}

static bool carries_constant(const Sys* s, const kv_problem_desc* d) {
    if (!s->d_b) return false;
    for (int j = 0; j < d->i; ++j)
        if (d->cols[j].is_fixed) return true;
    return false;
}

// The inner problem of the transpose dynamics (Sec. 4.1): one run per row of
// C (a sparse start vector, duplicate indices summed), the rows of
// E'^T = [E; constant row]^T as its projection, thresholds unused.
struct InnerDesc {
    kv_problem_desc d{};
    std::vector<kv_column> cols;
    std::vector<std::vector<int64_t>> ridx;
    std::vector<std::vector<double>> rval;
    std::vector<int64_t> crp, ccol;
    std::vector<double> cval, theta;
};

static void make_inner_desc(const Sys* s, const kv_problem_desc* d, bool taug, InnerDesc& in) {
    in.d = *d;
    in.cols.assign(d->o, kv_column{});
    in.ridx.assign(d->o, {});
    in.rval.assign(d->o, {});
    for (int r = 0; r < d->o; ++r) {
        std::vector<std::pair<int64_t, double>> e;
        for (int64_t q = d->c_row_ptr[r]; q < d->c_row_ptr[r + 1]; ++q) e.emplace_back(d->c_col[q], d->c_val[q]);
        std::sort(e.begin(), e.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        for (auto& pr : e) {
            if (!in.ridx[r].empty() && in.ridx[r].back() == pr.first) in.rval[r].back() += pr.second;
            else {
                in.ridx[r].push_back(pr.first);
                in.rval[r].push_back(pr.second);
            }
        }
        kv_column& c = in.cols[r];
        c.kind = KV_COL_SPARSE;
        c.zlo = c.zhi = 1.0;
        c.nnz = (int64_t)in.ridx[r].size();
        c.idx = in.ridx[r].data();
        c.val = in.rval[r].data();
    }
    in.crp.assign(1, 0);
    const int64_t n = s->n;
    for (int j = 0; j < d->i; ++j) {
        const kv_column& c = d->cols[j];
        if (c.kind == KV_COL_BOX) {
            const int64_t nx = s->dims[0], ny = s->dims[1];
            for (int64_t z = c.box_lo[2]; z < (s->ndim >= 3 ? c.box_hi[2] : 1); ++z)
                for (int64_t y = c.box_lo[1]; y < (s->ndim >= 2 ? c.box_hi[1] : 1); ++y)
                    for (int64_t x = c.box_lo[0]; x < c.box_hi[0]; ++x) {
                        in.ccol.push_back((z * ny + y) * nx + x);
                        in.cval.push_back(c.value);
                    }
        } else if (c.kind == KV_COL_SPARSE) {
            std::vector<std::pair<int64_t, double>> e;
            for (int64_t q = 0; q < c.nnz; ++q) e.emplace_back(c.idx[q], c.val[q]);
            std::sort(e.begin(), e.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
            for (auto& pr : e) {
                in.ccol.push_back(pr.first);
                in.cval.push_back(pr.second);
            }
        } else {
            for (int64_t q = 0; q < n; ++q)
                if (c.dense[q] != 0.0) {
                    in.ccol.push_back(q);
                    in.cval.push_back(c.dense[q]);
                }
        }
        if (taug && c.is_fixed) {
            in.ccol.push_back(n);  // the constant variable's entry of E_j
            in.cval.push_back(1.0);
        }
        in.crp.push_back((int64_t)in.ccol.size());
    }
    in.theta.assign(d->i, INFINITY);
    in.d.i = d->o;
    in.d.cols = in.cols.data();
    in.d.o = d->i;
    in.d.c_row_ptr = in.crp.data();
    in.d.c_col = in.ccol.data();
    in.d.c_val = in.cval.data();
    in.d.theta = in.theta.data();
    in.d.simulate = KV_SIM_FORWARD;
    if (in.d.method == KV_AUTO) in.d.method = (s->symmetric && !taug) ? KV_LANCZOS : KV_ARNOLDI;
}

static int vectors_needed(const Sys* s, const Prob* p) {
    int nv = 0;
    for (int j = 0; j < p->i; ++j) {
        int need = 0;
        if (p->method[j] == KV_LANCZOS) need = (s->kind == 0 && !p->fused && !p->fused64) ? 2 : 3;
        else need = p->m + 1;
        nv = std::max(nv, need);
    }
    return nv;
}

static void free_prob(Prob* p) {
    for (void* q : p->allocs) p->ctx->arena.free(q);
    p->allocs.clear();
    if (p->done_ev) cudaEventDestroy(p->done_ev);
    p->done_ev = nullptr;
}

static size_t bytes_core(const Sys* s, const kv_problem_desc* d, int precision, const BuildOpts& bo) {
    Prob tmp;
    tmp.sys = s;
    tmp.i = d->i;
    tmp.o = d->o;
    tmp.m = d->krylov_m;
    tmp.steps = d->steps;
    tmp.prec = precision;
    tmp.flags = d->flags;
    plan_methods(s, d, &tmp, bo);
    tmp.fused = !(d->flags & KV_FLAG_TWO_PASS) && fused_tma_supported(&tmp);
    tmp.fused64 = !(d->flags & KV_FLAG_TWO_PASS) && fused64_supported(&tmp);
    const int64_t N = s->n + (std::count(tmp.aug.begin(), tmp.aug.end(), 1) ? 1 : 0);
    const int nv = vectors_needed(s, &tmp);
    tmp.N = N;
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t t = 0;
    t += r256((size_t)nv * N * elem_size(precision) * vector_sets(s, d->i));
    if (s->kind == 1) t += r256((size_t)d->i * 4) + r256((size_t)d->i * 4) + r256(d->i * csr_arnoldi_dev_bytes());
    t += r256((size_t)d->i * d->o * (d->steps + 1) * sizeof(double));  // basis (Eq. memory_basis)
    t += 2 * r256((size_t)d->o * (d->steps + 1) * sizeof(double));      // lo, hi
    t += r256((size_t)d->i * (d->krylov_m + 1) * d->krylov_m * sizeof(double));
    t += r256((size_t)d->i * d->o * d->krylov_m * sizeof(double));
    t += r256((size_t)d->i * sizeof(ColState));
    t += r256((size_t)reduce_slots_needed(&tmp) * sizeof(double)) + 256;
    t += r256((size_t)(d->o + 1) * 8) + 2 * r256((size_t)d->c_row_ptr[d->o] * 8) + r256((size_t)d->o * 8);
    t += 3 * r256((size_t)d->i * 8) + 2 * 256;
    t += r256((size_t)d->i * 8) + r256((size_t)d->i * (d->steps + 1) * 8);  // error bound, its integrand
    t += r256(bounds_scratch_doubles(d->i, d->o, d->steps) * 8);
    if (needs_large_expm(d->krylov_m, d->expm_mode))
        t += r256(large_expm_scratch_doubles(d->krylov_m, d->steps) * 8 *
                  large_expm_batch(d->krylov_m, d->steps, d->i));
    for (int j = 0; j < d->i; ++j) {
        const kv_column& c = d->cols[j];
        if (c.kind == KV_COL_SPARSE) t += r256((size_t)(c.nnz + 1) * 8) * 2;
        if (c.kind == KV_COL_DENSE) t += r256((size_t)N * 8);
    }
    if (bo.brow) t += r256(((size_t)d->i * row_dot_blocks() + d->i) * 8);
    if (s->kind == 1) t += r256(csr_xi_bytes(&tmp));
    return t;
}

int kv_problem_bytes(const kv_sys* s, const kv_problem_desc* d, int precision, size_t* bytes) {
    if (!s || !d || !bytes) return fail(KV_EINVAL, "kv_problem_bytes: NULL argument");
    int rc = resolve_precision(s, d, precision, &precision);
    if (rc) return rc;
    rc = validate(s, d, precision);
    if (rc) return rc;
    if (!runs_transposed(d)) {
        *bytes = bytes_core(s, d, precision, BuildOpts{});
        return KV_OK;
    }
    const bool taug = carries_constant(s, d);
    InnerDesc in;
    make_inner_desc(s, d, taug, in);
    BuildOpts bo;
    bo.trans_runs = true;
    bo.trans_aug = taug ? 1 : 0;
    bo.brow = taug ? s->d_b : nullptr;
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t t = bytes_core(s, &in.d, precision, bo);
    const size_t S = (size_t)d->steps + 1;
    t += r256((size_t)d->i * d->o * S * 8) + 2 * r256((size_t)d->o * S * 8) + r256((size_t)d->o * 8) +
         3 * r256((size_t)d->i * 8) + 2 * 256 + r256(bounds_scratch_doubles(d->i, d->o, d->steps) * 8);
    if (s->kind == 1 && !s->symmetric && !s->d_rpT)  // A^T, built on first use
        t += r256((size_t)(s->n + 1) * 8) + r256((size_t)s->nnz * 4) + r256((size_t)s->nnz * elem_size(precision));
    *bytes = t;
    return KV_OK;
}

// Fills and allocates p (fresh) for problem d on system s; on failure p's
// device memory is released (the caller deletes p).
static int prob_build(Ctx* c, Prob* p, const Sys* s, const kv_problem_desc* d, int precision, const BuildOpts& bo) {
    int rc = KV_OK;
    p->ctx = c;
    p->sys = s;
    p->prec = precision;
    p->i = d->i;
    p->o = d->o;
    p->m = d->krylov_m;
    p->steps = d->steps;
    p->dt = d->dt;
    p->expm_mode = d->expm_mode;
    p->batched = d->batched;
    p->flags = d->flags;
    p->err_target = d->err_target > 0.0 ? d->err_target : 0.0;
    p->trans_runs = bo.trans_runs;
    p->d_brow = bo.brow;
    plan_methods(s, d, p, bo);
    p->fused = !(d->flags & KV_FLAG_TWO_PASS) && fused_tma_supported(p);
    p->fused64 = !(d->flags & KV_FLAG_TWO_PASS) && fused64_supported(p);
    p->N = s->n + (std::count(p->aug.begin(), p->aug.end(), 1) ? 1 : 0);
    p->nvec = vectors_needed(s, p);
    p->cols.assign(d->cols, d->cols + d->i);
    const int64_t S = d->steps + 1;
    const int64_t cnnz = d->c_row_ptr[d->o];
    p->c_nnz = cnnz;
#define TRY(x)               \
    do {                     \
        rc = (x);            \
        if (rc) goto failed; \
    } while (0)
    {
        p->nsets = vector_sets(s, p->i);
        size_t vec_bytes = 0;  // nvec x N x element size x sets, checked for overflow
        if (__builtin_mul_overflow((size_t)p->nvec, (size_t)p->N, &vec_bytes) ||
            __builtin_mul_overflow(vec_bytes, (size_t)elem_size(precision), &vec_bytes) ||
            __builtin_mul_overflow(vec_bytes, (size_t)p->nsets, &vec_bytes))
            TRY(fail(KV_ENOMEM, "Krylov vectors: size overflows"));
        TRY(dalloc(p, (char**)&p->d_vec, vec_bytes));
        if (s->kind == 1) {
            TRY(dalloc(p, &p->d_counters, (size_t)p->i));
            TRY(dalloc(p, &p->d_aug, (size_t)p->i));
            TRY(dalloc(p, (char**)&p->d_arnoldi, (size_t)p->i * csr_arnoldi_dev_bytes()));
            KV_CHECK_CUDA(cudaMemsetAsync(p->d_counters, 0, (size_t)p->i * sizeof(unsigned), c->stream));
            KV_CHECK_CUDA(cudaMemsetAsync(p->d_arnoldi, 0, (size_t)p->i * csr_arnoldi_dev_bytes(), c->stream));
            TRY(upload(c, p->d_aug, p->aug.data(), (size_t)p->i * sizeof(int)));
        }
        TRY(dalloc(p, &p->d_basis, (size_t)p->i * p->o * S));
        TRY(dalloc(p, &p->d_lo, (size_t)p->o * S));
        TRY(dalloc(p, &p->d_hi, (size_t)p->o * S));
        TRY(dalloc(p, &p->d_H, (size_t)p->i * (p->m + 1) * p->m));
        TRY(dalloc(p, &p->d_P, (size_t)p->i * p->o * p->m));
        TRY(dalloc(p, &p->d_state, (size_t)p->i));
        p->red_slots = (int)reduce_slots_needed(p);
        TRY(dalloc(p, &p->red.partials, (size_t)p->red_slots));
        TRY(dalloc(p, &p->red.counter, 1));
        TRY(dalloc(p, &p->d_crp, (size_t)p->o + 1));
        TRY(dalloc(p, &p->d_ccol, (size_t)std::max<int64_t>(cnnz, 1)));
        TRY(dalloc(p, &p->d_cval, (size_t)std::max<int64_t>(cnnz, 1)));
        TRY(dalloc(p, &p->d_theta, (size_t)p->o));
        TRY(dalloc(p, &p->d_zlo, (size_t)p->i));
        TRY(dalloc(p, &p->d_zhi, (size_t)p->i));
        TRY(dalloc(p, &p->d_zstar, (size_t)p->i));
        TRY(dalloc(p, &p->d_ystar, 1));
        TRY(dalloc(p, &p->d_viol, 1));
        TRY(dalloc(p, &p->d_err, (size_t)p->i));
        if (bounds_scratch_doubles(p->i, p->o, p->steps))
            TRY(dalloc(p, &p->d_bpart, bounds_scratch_doubles(p->i, p->o, p->steps)));
        TRY(dalloc(p, &p->d_hlast, (size_t)p->i * S));
        if (needs_large_expm(p->m, p->expm_mode))
            TRY(dalloc(p, &p->d_lx, large_expm_scratch_doubles(p->m, p->steps) * large_expm_batch(p->m, p->steps, p->i)));
        if (p->d_brow) {
            const size_t nrd = (size_t)p->i * row_dot_blocks() + p->i;  // partials, then tickets
            TRY(dalloc(p, &p->d_rowdot, nrd));
            KV_CHECK_CUDA(cudaMemsetAsync(p->d_rowdot, 0, nrd * 8, c->stream));
        }
        TRY(upload(c, p->d_crp, d->c_row_ptr, (size_t)(p->o + 1) * 8));
        TRY(upload(c, p->d_ccol, d->c_col, (size_t)cnnz * 8));
        TRY(upload(c, p->d_cval, d->c_val, (size_t)cnnz * 8));
        TRY(upload(c, p->d_theta, d->theta, (size_t)p->o * 8));
        std::vector<double> zl(p->i), zh(p->i);
        for (int j = 0; j < p->i; ++j) {
            zl[j] = d->cols[j].zlo;
            zh[j] = d->cols[j].zhi;
        }
        TRY(upload(c, p->d_zlo, zl.data(), (size_t)p->i * 8));
        TRY(upload(c, p->d_zhi, zh.data(), (size_t)p->i * 8));
        KV_CHECK_CUDA(cudaMemsetAsync(p->red.counter, 0, sizeof(unsigned), c->stream));
        KV_CHECK_CUDA(cudaMemsetAsync(p->d_H, 0, (size_t)p->i * (p->m + 1) * p->m * 8, c->stream));
        KV_CHECK_CUDA(cudaMemsetAsync(p->d_P, 0, (size_t)p->i * p->o * p->m * 8, c->stream));
        p->d_sidx.assign(p->i, nullptr);
        p->sidx_n.assign(p->i, 0);
        p->d_sval.assign(p->i, nullptr);
        p->d_dense.assign(p->i, nullptr);
        for (int j = 0; j < p->i; ++j) {
            const kv_column& col = d->cols[j];
            kv_column& hc = p->cols[j];
            hc.idx = nullptr;
            hc.val = nullptr;
            hc.dense = nullptr;
            if (col.kind == KV_COL_SPARSE) {
                const bool cst = p->aug[j] && !p->trans_runs;  // the constant entry of E_j is 1
                const int64_t nn = col.nnz + (cst ? 1 : 0);
                std::vector<int64_t> ix(col.idx, col.idx + col.nnz);
                std::vector<double> vv(col.val, col.val + col.nnz);
                if (cst) {
                    ix.push_back(s->n);
                    vv.push_back(1.0);
                }
                TRY(dalloc(p, &p->d_sidx[j], (size_t)std::max<int64_t>(nn, 1)));
                TRY(dalloc(p, &p->d_sval[j], (size_t)std::max<int64_t>(nn, 1)));
                TRY(upload(c, p->d_sidx[j], ix.data(), (size_t)nn * 8));
                TRY(upload(c, p->d_sval[j], vv.data(), (size_t)nn * 8));
                p->sidx_n[j] = nn;
                KV_CHECK_CUDA(cudaStreamSynchronize(c->stream));  // host vectors go out of scope
            } else if (col.kind == KV_COL_DENSE) {
                TRY(dalloc(p, &p->d_dense[j], (size_t)p->N));
                TRY(upload(c, p->d_dense[j], col.dense, (size_t)s->n * 8));
                if (p->N > s->n) {
                    static const double one = 1.0, zero = 0.0;
                    TRY(upload(c, p->d_dense[j] + s->n, (p->aug[j] && !p->trans_runs) ? &one : &zero, 8));
                }
            }
        }
        if (s->kind == 1) {
            if (const size_t xb = csr_xi_bytes(p)) TRY(dalloc(p, (char**)&p->d_xi, xb));
            TRY(csr_autotune(p));
        }
        if (cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming) != cudaSuccess) {
            rc = fail(KV_ECUDA, "event creation failed");
            goto failed;
        }
        KV_CHECK_CUDA(cudaStreamSynchronize(c->stream));
    }
#undef TRY
    return KV_OK;
failed:
    cudaStreamSynchronize(c->stream);
    free_prob(p);
    return rc;
}

// The transpose dynamics (Sec. 4.1): an inner problem with one run per row of
// C on A^T (A'^T when a column carries the constant), projected by E'^T, and
// this outer problem holding the external thresholds, box and outputs.
static int build_transposed(kv_ctx* c, kv_prob** out, const Sys* s, const kv_problem_desc* d, int precision) {
    const bool taug = carries_constant(s, d);
    int rc = KV_OK;
    if (s->kind == 1 && !s->symmetric) {
        rc = csr_build_transpose(const_cast<Sys*>(s));
        if (rc) return rc;
    }
    InnerDesc in;
    make_inner_desc(s, d, taug, in);
    Sys* view = new (std::nothrow) Sys(*s);
    Prob* inner = new (std::nothrow) Prob();
    kv_prob* p = new (std::nothrow) kv_prob();
    if (!view || !inner || !p) {
        delete view;
        delete inner;
        delete p;
        return fail(KV_ENOMEM, "host allocation");
    }
    if (s->kind == 1 && !s->symmetric) {
        view->d_rp = s->d_rpT;
        view->d_col = s->d_colT;
        view->d_val = s->d_valT;
    }
    view->d_rpT = nullptr;
    view->d_colT = nullptr;
    view->d_valT = nullptr;
    view->d_b = nullptr;  // the rows of A'^T but the last carry no b; the last is k_row_dot's
    BuildOpts bo;
    bo.trans_runs = true;
    bo.trans_aug = taug ? 1 : 0;
    bo.brow = taug ? s->d_b : nullptr;
    rc = prob_build(c, inner, view, &in.d, precision, bo);
    if (rc) {
        delete inner;
        delete view;
        delete p;
        return rc;
    }
    p->ctx = c;
    p->sys = s;
    p->prec = precision;
    p->i = d->i;
    p->o = d->o;
    p->m = d->krylov_m;
    p->steps = d->steps;
    p->dt = d->dt;
    p->expm_mode = d->expm_mode;
    p->flags = d->flags;
    p->err_target = inner->err_target;
    p->inner = inner;
    p->view = view;
    p->cols.assign(d->cols, d->cols + d->i);  // boxes only: the caller's arrays are not kept
    for (kv_column& hc : p->cols) {
        hc.idx = nullptr;
        hc.val = nullptr;
        hc.dense = nullptr;
    }
    const int64_t S = d->steps + 1;
#define TRY(x)               \
    do {                     \
        rc = (x);            \
        if (rc) goto failed; \
    } while (0)
    {
        TRY(dalloc(p, &p->d_basis, (size_t)p->i * p->o * S));
        TRY(dalloc(p, &p->d_lo, (size_t)p->o * S));
        TRY(dalloc(p, &p->d_hi, (size_t)p->o * S));
        TRY(dalloc(p, &p->d_theta, (size_t)p->o));
        TRY(dalloc(p, &p->d_zlo, (size_t)p->i));
        TRY(dalloc(p, &p->d_zhi, (size_t)p->i));
        TRY(dalloc(p, &p->d_zstar, (size_t)p->i));
        TRY(dalloc(p, &p->d_ystar, 1));
        TRY(dalloc(p, &p->d_viol, 1));
        if (bounds_scratch_doubles(p->i, p->o, p->steps))
            TRY(dalloc(p, &p->d_bpart, bounds_scratch_doubles(p->i, p->o, p->steps)));
        TRY(upload(c, p->d_theta, d->theta, (size_t)p->o * 8));
        std::vector<double> zl(p->i), zh(p->i);
        for (int j = 0; j < p->i; ++j) {
            zl[j] = d->cols[j].zlo;
            zh[j] = d->cols[j].zhi;
        }
        TRY(upload(c, p->d_zlo, zl.data(), (size_t)p->i * 8));
        TRY(upload(c, p->d_zhi, zh.data(), (size_t)p->i * 8));
        if (cudaEventCreateWithFlags(&p->done_ev, cudaEventDisableTiming) != cudaSuccess) {
            rc = fail(KV_ECUDA, "event creation failed");
            goto failed;
        }
        KV_CHECK_CUDA(cudaStreamSynchronize(c->stream));
    }
#undef TRY
    *out = p;
    return KV_OK;
failed:
    cudaStreamSynchronize(c->stream);
    free_prob(inner);
    delete inner;
    delete view;
    free_prob(p);
    delete p;
    return rc;
}

int kv_problem(kv_ctx* c, kv_prob** out, const kv_sys* s, const kv_problem_desc* d, int precision) {
    if (!c || !out || !s) return fail(KV_EINVAL, "kv_problem: NULL argument");
    *out = nullptr;
    if (s->ctx != c) return fail(KV_EINVAL, "kv_problem: system belongs to another context");
    if (!d) return fail(KV_EINVAL, "kv_problem: NULL argument");
    int rc = resolve_precision(s, d, precision, &precision);
    if (rc) return rc;
    rc = validate(s, d, precision);
    if (rc) return rc;
    KV_WITH_DEVICE(c->device);
    if (runs_transposed(d)) return build_transposed(c, out, s, d, precision);
    kv_prob* p = new (std::nothrow) kv_prob();
    if (!p) return fail(KV_ENOMEM, "host allocation");
    rc = prob_build(c, p, s, d, precision, BuildOpts{});
    if (rc) {
        delete p;
        return rc;
    }
    *out = p;
    return KV_OK;
}

#ifdef KV_DEBUG
int kv_debug_set_c_col(kv_prob* p, int64_t e, int64_t value) {
    if (!p) return fail(KV_EINVAL, "kv_debug_set_c_col: NULL problem");
    if (p->inner) return fail(KV_EINVAL, "kv_debug_set_c_col: forward problems only");
    KV_WITH_DEVICE(p->ctx->device);
    KV_CHECK_CUDA(cudaStreamSynchronize(p->ctx->stream));
    int64_t cnnz = 0;
    KV_CHECK_CUDA(cudaMemcpy(&cnnz, p->d_crp + p->o, sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (e < 0 || e >= cnnz) return fail(KV_EINVAL, "kv_debug_set_c_col: entry %lld of %lld", (long long)e, (long long)cnnz);
    KV_CHECK_CUDA(cudaMemcpy(p->d_ccol + e, &value, sizeof(int64_t), cudaMemcpyHostToDevice));
    return KV_OK;
}
#endif

int kv_problem_precision(const kv_prob* p, int32_t* precision) {
    if (!p || !precision) return fail(KV_EINVAL, "kv_problem_precision: NULL argument");
    *precision = p->prec;
    return KV_OK;
}

int kv_problem_runs(const kv_prob* p, int32_t* runs, int32_t* transposed) {
    if (!p || !runs || !transposed) return fail(KV_EINVAL, "kv_problem_runs: NULL argument");
    *runs = p->inner ? p->inner->i : p->i;
    *transposed = p->inner ? 1 : 0;
    return KV_OK;
}

int kv_prob_destroy(kv_prob* p) {
    if (!p) return KV_OK;
    ::kv::DeviceGuard kv_device_guard_(p->ctx->device);
    cudaStreamSynchronize(p->ctx->stream);
    if (p->inner) {
        free_prob(p->inner);
        delete p->inner;
        delete p->view;
    }
    free_prob(p);
    delete p;
    return KV_OK;
}

static int run_column(Prob* p, int j) {
    const Sys* s = p->sys;
    const size_t es = elem_size(p->prec);
    char* base = (char*)p->d_vec;
    auto vec = [&](int q) { return (void*)(base + (size_t)q * p->N * es); };
    int rc;
    const kv_column& c = p->cols[j];
    if (c.kind == KV_COL_BOX) {
        rc = launch_stencil_init_box(p, j, vec(0));
    } else {
        rc = c.kind == KV_COL_SPARSE ? launch_scatter(p, j, vec(0)) : launch_dense_to(p, j, vec(0));
        if (!rc) rc = launch_init_norm(p, j, vec(0));
    }
    if (rc) return rc;
    if (p->method[j] == KV_LANCZOS && s->kind == 0 && (p->fused || p->fused64)) {
        // alpha_0 (closed form for a box column, else one read pass), then
        // one fused pass per iteration over three rotating buffers
        if (c.kind != KV_COL_BOX) {
            rc = launch_stencil_alpha(p, j, 0, vec(0));
            if (rc) return rc;
        }
        for (int it = 0; it < p->m; ++it) {
            if (p->fused64)
                rc = launch_lanczos_fused64(p, j, it, vec(it % 3), vec((it + 2) % 3), vec((it + 1) % 3));
            else
                rc = launch_lanczos_fused(p, j, it, vec(it % 3), vec((it + 2) % 3), vec((it + 1) % 3));
            if (!rc) rc = launch_project(p, j, 1, vec((it + 1) % 3), 0, it + 1);
            if (!rc && is_checkpoint(p, it + 1)) rc = launch_error_check(p, j, 1, it + 1);
            if (rc) return rc;
        }
        return KV_OK;
    }
    if (p->method[j] == KV_LANCZOS && s->kind == 0) {
        for (int it = 0; it < p->m; ++it) {
            void* B = vec(it & 1);
            void* A = vec((it + 1) & 1);
            rc = launch_stencil_alpha(p, j, it, B);
            if (!rc) rc = launch_stencil_update(p, j, it, B, A);
            if (!rc) rc = launch_project(p, j, 1, A, 0, it + 1);
            if (!rc && is_checkpoint(p, it + 1)) rc = launch_error_check(p, j, 1, it + 1);
            if (rc) return rc;
        }
        return KV_OK;
    }
    return fail(KV_EINVAL, "grid systems run Lanczos only");
}

// CSR: initial vectors of every column into slot 0 of its own vector set,
// then each run of consecutive same-method columns as one set of launches
// (grid.y = column).
static int run_csr(Prob* p) {
    const size_t es = elem_size(p->prec);
    const size_t set_bytes = (size_t)p->nvec * p->N * es;
    auto set = [&](int j) { return (void*)((char*)p->d_vec + (size_t)j * set_bytes); };
    int rc;
    for (int j = 0; j < p->i; ++j) {
        const kv_column& c = p->cols[j];
        rc = c.kind == KV_COL_SPARSE ? launch_scatter(p, j, set(j)) : launch_dense_to(p, j, set(j));
        if (!rc) rc = launch_init_norm(p, j, set(j));
        if (rc) return rc;
    }
    for (int j0 = 0; j0 < p->i;) {
        int j1 = j0;
        while (j1 < p->i && p->method[j1] == p->method[j0]) ++j1;
        rc = launch_csr_columns(p, j0, j1 - j0, set(j0), p->method[j0] == KV_LANCZOS);
        if (rc) return rc;
        j0 = j1;
    }
    return KV_OK;
}

// The Krylov runs of p, the exponentials and basis rows, the error bounds.
static int enqueue_runs(Prob* p) {
    int rc = KV_OK;
    if (p->sys->kind == 1) {
        rc = run_csr(p);
        if (rc) return rc;
    } else {
        for (int j = 0; j < p->i; ++j) {
            rc = run_column(p, j);
            if (rc) return rc;
        }
    }
    rc = launch_expm_basis(p);
    if (!rc) rc = launch_error_final(p);
    return rc;
}

int kv_enqueue(kv_prob* p) {
    if (!p) return fail(KV_EINVAL, "kv_enqueue: NULL problem");
    KV_WITH_DEVICE(p->ctx->device);
    int rc = KV_OK;
    if (p->inner) {
        // transpose dynamics: basis rows per output row, then transposed
        rc = enqueue_runs(p->inner);
        if (!rc) rc = launch_basis_transpose(p->inner, p->d_basis, p->ctx->stream);
    } else {
        rc = enqueue_runs(p);
    }
    if (rc) return rc;
    rc = launch_bounds(p);
    if (rc) return rc;
    KV_CHECK_CUDA(cudaEventRecord(p->done_ev, p->ctx->stream));
    p->ran = true;
    return KV_OK;
}

int kv_fetch(kv_prob* p, kv_result* r) {
    if (!p || !r || !r->lo || !r->hi) return fail(KV_EINVAL, "kv_fetch: NULL argument");
    KV_WITH_DEVICE(p->ctx->device);
    int rc = KV_OK;
    KV_CHECK_CUDA(cudaEventSynchronize(p->done_ev));
    const size_t S = (size_t)p->steps + 1;
    KV_CHECK_CUDA(cudaMemcpy(r->lo, p->d_lo, (size_t)p->o * S * 8, cudaMemcpyDeviceToHost));
    KV_CHECK_CUDA(cudaMemcpy(r->hi, p->d_hi, (size_t)p->o * S * 8, cudaMemcpyDeviceToHost));
    if (r->basis) KV_CHECK_CUDA(cudaMemcpy(r->basis, p->d_basis, (size_t)p->i * p->o * S * 8, cudaMemcpyDeviceToHost));
    const Prob* q = p->inner ? p->inner : p;  // the Krylov runs
    if (r->H) KV_CHECK_CUDA(cudaMemcpy(r->H, q->d_H, (size_t)q->i * (q->m + 1) * q->m * 8, cudaMemcpyDeviceToHost));
    if (r->P) KV_CHECK_CUDA(cudaMemcpy(r->P, q->d_P, (size_t)q->i * q->o * q->m * 8, cudaMemcpyDeviceToHost));
    std::vector<ColState> st(q->i);
    KV_CHECK_CUDA(cudaMemcpy(st.data(), q->d_state, (size_t)q->i * sizeof(ColState), cudaMemcpyDeviceToHost));
    int status = 0;
    for (int j = 0; j < q->i; ++j) {
        if (r->beta0) r->beta0[j] = st[j].beta0;
        if (r->m_used) r->m_used[j] = st[j].m_used;
        status |= st[j].status;
    }
    int key = 0;
    KV_CHECK_CUDA(cudaMemcpy(&key, p->d_viol, sizeof(int), cudaMemcpyDeviceToHost));
    if (key == 0x7f7f7f7f) {
        r->first_violation_step = -1;
        r->violation_row = -1;
        r->y_star = 0.0;
    } else {
        r->first_violation_step = key / p->o;
        r->violation_row = key % p->o;
        KV_CHECK_CUDA(cudaMemcpy(&r->y_star, p->d_ystar, sizeof(double), cudaMemcpyDeviceToHost));
        if (r->z_star) KV_CHECK_CUDA(cudaMemcpy(r->z_star, p->d_zstar, (size_t)p->i * 8, cudaMemcpyDeviceToHost));
    }
    if (r->err_bound) KV_CHECK_CUDA(cudaMemcpy(r->err_bound, q->d_err, (size_t)q->i * 8, cudaMemcpyDeviceToHost));
    if (status & KV_ST_TIMEOUT) return fail(KV_ETIMEOUT, "a device-side wait gave up (status %d)", status);
    if (status & KV_ST_INDEX)
        return fail(KV_EINVAL, "a device-side bounds check skipped an index outside its vector (status %d): the "
                    "results are incomplete", status);
    if (status & KV_ST_NONFINITE)
        return fail(KV_EINVAL, "a Krylov scalar (the norm of a column, alpha or beta) is not finite (status %d): "
                    "the system or the initial set holds a NaN or overflows", status);
    if (status & KV_ST_SCALING)
        return fail(KV_EINVAL, "an exponential of H needed more squarings than the operator's norm bound allowed "
                    "(status %d)", status);
    return KV_OK;
}

int kv_check_polytope(kv_prob* p, const kv_polytope* unsafe, const kv_polytope* init, double tol, kv_lp_result* r) {
    if (!p || !unsafe || !r || !r->margin || !r->status) return fail(KV_EINVAL, "kv_check_polytope: NULL argument");
    if (!p->ran) return fail(KV_EINVAL, "kv_check_polytope: the problem has not run");
    const int qu = unsafe->rows, qi = init ? init->rows : 0;
    if (qu < 1 || !unsafe->a || !unsafe->rhs) return fail(KV_EINVAL, "kv_check_polytope: the unsafe set needs rows");
    if (qi < 0 || (qi > 0 && (!init->a || !init->rhs))) return fail(KV_EINVAL, "kv_check_polytope: bad initial rows");
    if (std::isnan(tol)) return fail(KV_EINVAL, "kv_check_polytope: tol is NaN");
    const int i = p->i, o = p->o;
    const int64_t S = (int64_t)p->steps + 1;
    for (int j = 0; j < i; ++j)
        if (!std::isfinite(p->cols[j].zlo) || !std::isfinite(p->cols[j].zhi))
            return fail(KV_EINVAL, "kv_check_polytope: column %d has an infinite box", j);
    // unsafe rows scaled to unit norm (the same half-spaces)
    std::vector<double> U((size_t)qu * o), v(qu);
    for (int u = 0; u < qu; ++u) {
        double nr = 0.0;
        for (int c = 0; c < o; ++c) nr += unsafe->a[(size_t)u * o + c] * unsafe->a[(size_t)u * o + c];
        nr = std::sqrt(nr);
        if (!(nr > 0.0) || !std::isfinite(nr) || !std::isfinite(unsafe->rhs[u]))
            return fail(KV_EINVAL, "kv_check_polytope: unsafe row %d is zero or not finite", u);
        for (int c = 0; c < o; ++c) U[(size_t)u * o + c] = unsafe->a[(size_t)u * o + c] / nr;
        v[u] = unsafe->rhs[u] / nr;
    }
    for (int64_t q = 0; q < (int64_t)qi * (i + 1); ++q) {
        const double x = q < (int64_t)qi * i ? init->a[q] : init->rhs[q - (int64_t)qi * i];
        if (!std::isfinite(x)) return fail(KV_EINVAL, "kv_check_polytope: initial rows not finite");
    }
    const int m = qu + qi + 2 * i;
    int dev_max = 0;
    KV_CHECK_CUDA(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->ctx->device));
    if (lp_smem_bytes(i, m) > (size_t)dev_max)
        return fail(KV_EINVAL, "kv_check_polytope: the LP (i = %d, %d constraints) needs %zu bytes of shared memory, "
                    "the device allows %d", i, m, lp_smem_bytes(i, m), dev_max);
    KV_WITH_DEVICE(p->ctx->device);
    int rc = KV_OK;
    Ctx* c = p->ctx;
    // one arena block: U, v, Iz, iota, margin, zx, yx (doubles), status (ints)
    const size_t nd = (size_t)qu * o + qu + (size_t)qi * i + qi + S + (size_t)S * i + (size_t)S * o;
    char* buf = (char*)c->arena.alloc(nd * 8 + (size_t)S * 4 + 4);
    if (!buf) return fail(KV_ENOMEM, "kv_check_polytope: device pool exhausted (%zu bytes)", nd * 8 + (size_t)S * 4 + 4);
    double* dU = (double*)buf;
    double* dv = dU + (size_t)qu * o;
    double* dIz = dv + qu;
    double* diota = dIz + (size_t)qi * i;
    double* dmargin = diota + qi;
    double* dzx = dmargin + S;
    double* dyx = dzx + (size_t)S * i;
    int* dstatus = (int*)(dyx + (size_t)S * o);
    int* dzflag = dstatus + S;  // the initial set's emptiness, from the first launch
    std::vector<double> zx((size_t)S * i);
    auto run = [&]() -> int {
        int e = upload(c, dU, U.data(), U.size() * 8);
        if (!e) e = upload(c, dv, v.data(), v.size() * 8);
        if (!e && qi) e = upload(c, dIz, init->a, (size_t)qi * i * 8);
        if (!e && qi) e = upload(c, diota, init->rhs, (size_t)qi * 8);
        if (!e) KV_CHECK_CUDA(cudaStreamWaitEvent(c->stream, p->done_ev, 0));
        if (!e) e = launch_step_lp(p, dU, dv, qu, dIz, diota, qi, m, dmargin, dstatus, dzx, dyx, dzflag);
        if (e) return e;
        KV_CHECK_CUDA(cudaMemcpyAsync(r->margin, dmargin, (size_t)S * 8, cudaMemcpyDeviceToHost, c->stream));
        KV_CHECK_CUDA(cudaMemcpyAsync(r->status, dstatus, (size_t)S * 4, cudaMemcpyDeviceToHost, c->stream));
        KV_CHECK_CUDA(cudaMemcpyAsync(zx.data(), dzx, zx.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        KV_CHECK_CUDA(cudaStreamSynchronize(c->stream));
        r->first_violation_step = -1;
        for (int64_t k = 0; k < S; ++k)
            if (r->status[k] == KV_LP_OPTIMAL && r->margin[k] <= tol) {
                r->first_violation_step = (int32_t)k;
                break;
            }
        if (r->z) std::copy(zx.begin(), zx.end(), r->z);
        const int64_t kv = r->first_violation_step;
        if (kv >= 0) {
            if (r->z_star) std::copy(zx.begin() + kv * i, zx.begin() + (kv + 1) * i, r->z_star);
            if (r->y_star) KV_CHECK_CUDA(cudaMemcpy(r->y_star, dyx + kv * o, (size_t)o * 8, cudaMemcpyDeviceToHost));
        }
        return KV_OK;
    };
    rc = run();
    cudaStreamSynchronize(c->stream);  // nothing in flight reads the block when it is freed
    c->arena.free(buf);
    return rc;
}

int kv_run(kv_prob* p, kv_result* r) {
    int rc = kv_enqueue(p);
    if (rc) return rc;
    return kv_fetch(p, r);
}

int kv_profile_enable(kv_ctx* c, int enable) {
    if (!c) return fail(KV_EINVAL, "kv_profile_enable: NULL ctx");
    ::kv::DeviceGuard kv_device_guard_(c->device);
    cudaStreamSynchronize(c->stream);
    clear_profile(c);
    c->profiling = enable != 0;
    return KV_OK;
}

int kv_profile_read(kv_ctx* c, const char* name, int64_t* launches, double* total_ms) {
    if (!c || !name || !launches || !total_ms) return fail(KV_EINVAL, "kv_profile_read: NULL argument");
    KV_WITH_DEVICE(c->device);
    KV_CHECK_CUDA(cudaStreamSynchronize(c->stream));
    int64_t n = 0;
    double t = 0.0;
    for (auto& r : c->recs) {
        if (r.name != name) continue;
        float ms = 0.f;
        KV_CHECK_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        n++;
        t += ms;
    }
    *launches = n;
    *total_ms = t;
    return KV_OK;
}

}  // extern "C"
