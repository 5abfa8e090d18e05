// k_stencil_tma.cu -- single-pass Lanczos iteration on the grid Laplacian
// (FP32 storage), with TMA-staged planes.
//
// One launch performs iteration j of the projected Lanczos loop (Alg. 3 with
// the Alg. 4 projection):
//     w = A v_j - alpha_j v_j - beta_j v_{j-1}           (written to a third buffer)
//     beta_{j+1}^2 = w . w,  alpha_{j+1} = (w . A w) / (w . w)
//     P[:, j+1] = C w / beta_{j+1}
// so alpha of the *next* iteration comes out of the same pass and every
// iteration reads v_j and v_{j-1} once and writes w once (12 bytes per grid
// point in FP32, the algorithmic minimum of a three-vector Lanczos step).
//
// Each CTA owns a 128 x 16 (x, y) tile and marches over a chunk of z planes.
// Per plane, one elected thread issues TMA tile loads (cp.async.bulk.tensor,
// completion counted on an mbarrier) of
//     v_j     with a 2-point halo in y (and 4 in x, the 16-byte TMA granule),
//     v_{j-1} with a 1-point halo in y,
// into a shared-memory ring two planes ahead of the compute.  TMA fills
// coordinates outside the grid with zeros, which is the Dirichlet-0 boundary.
// w is evaluated on the tile plus a 1-point halo ring (so A w of the interior
// needs no data from neighbouring CTAs) into a 3-plane ring; the interior of
// plane q = p - 1 is then finished: A w, the two dot products (error-free
// float accumulation, Dot2) and the store of w.  w is written to a buffer no
// CTA reads in this pass, so tiles never race on halos.
//
// Every mbarrier wait is bounded; on expiry the CTA sets the column's status
// word (reported as KV_ETIMEOUT), drains its own outstanding copies with a
// bounded wait and leaves.
#include <cuda.h>

#include "kv_internal.h"
#include "reduce.cuh"

namespace kv {

constexpr int FTX = 128, FTY = 16, FNT = 256;
constexpr int HX = 4;                  // x halo: one 16-byte TMA granule of floats
constexpr int BW = FTX + 2 * HX;       // 136: box width of both loads
constexpr int BH = FTY + 4;            // 20: v_j box height (2-row halo)
constexpr int AH = FTY + 2;            // 18: v_{j-1} box height (1-row halo)
constexpr int WW = FTX + 2, WH = FTY + 2;  // w region: tile + 1 halo
constexpr int DEPTH = 2;               // stages in flight
constexpr int RB = DEPTH + 2, RA = DEPTH;
constexpr int BBYTES = BW * BH * 4;    // 10880
constexpr int ABYTES = BW * AH * 4;    // 9792
constexpr int BSTRIDE = (BBYTES + 127) / 128 * 128;
constexpr int ASTRIDE = (ABYTES + 127) / 128 * 128;
constexpr int WSTRIDE = (WW * WH * 4 + 127) / 128 * 128;
constexpr int SMEM_MAIN = RB * BSTRIDE + RA * ASTRIDE + 3 * WSTRIDE;
constexpr int SMEM_TOTAL = SMEM_MAIN + 128 + 1024;  // + barriers + alignment slack
constexpr long WAIT_LIMIT = 1L << 22;

__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
    for (long it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(saddr(dst)),
        "l"((uint64_t)map), "r"(saddr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

struct FusedArgs {
    float* W;          // output buffer (w = unnormalised v_{j+1})
    StencilGeom g;
    int zc;            // z planes per CTA
    ColState* st;
    double* H;         // this column's (m+1) x m
    double* P;         // this column's o x m
    CDesc cd;
    int m, j;
    Reduce red;
};

template <bool FIRST>
__global__ void __launch_bounds__(FNT, 2) k_lanczos_fused_tma(const __grid_constant__ CUtensorMap mapB,
                                                             const __grid_constant__ CUtensorMap mapA,
                                                             FusedArgs a) {
    if (a.st->done) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float* sB = (float*)sm;
    float* sA = (float*)(sm + RB * BSTRIDE);
    float* sW = (float*)(sm + RB * BSTRIDE + RA * ASTRIDE);
    uint64_t* bars = (uint64_t*)(sm + SMEM_MAIN);  // DEPTH stage barriers + 1 prologue barrier
    __shared__ double shred[FNT / 32];
    __shared__ int flag, abort_flag;

    const int t = threadIdx.x;
    const StencilGeom& g = a.g;
    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int z0 = blockIdx.z * a.zc;
    const int z1 = (int)min((int64_t)z0 + a.zc, g.nz);
    const int p0 = z0 - 1, pend = z1;  // w planes computed: p0 .. pend

    // coefficients of w = ax (B_l + B_r) + ay (B_d + B_u) + az (B_b + B_f) + bc B_c + ba A
    const double sj = a.st->s[a.j];
    const double alpha = a.H[(int64_t)a.j * a.m + a.j];
    const float ax = (float)(sj * g.kx), ay = (float)(sj * g.ky), az = (float)(sj * g.kz);
    const float bc = (float)(sj * (g.kc - alpha));
    const float ba = FIRST ? 0.f : (float)(-a.H[(int64_t)a.j * a.m + (a.j - 1)] * a.st->s[a.j - 1]);
    const float kx = (float)g.kx, ky = (float)g.ky, kz = (float)g.kz, kc = (float)g.kc;

    auto bslot = [&](int plane) { return sB + (size_t)(((plane % RB) + RB) % RB) * (BSTRIDE / 4); };
    auto aslot = [&](int plane) { return sA + (size_t)(((plane % RA) + RA) % RA) * (ASTRIDE / 4); };
    auto wslot = [&](int plane) { return sW + (size_t)(((plane % 3) + 3) % 3) * (WSTRIDE / 4); };
    const unsigned stage_bytes = BBYTES + (FIRST ? 0u : (unsigned)ABYTES);

    auto issue_stage = [&](int p) {  // B plane p+1, A plane p -> stage barrier of p
        uint64_t* bar = bars + ((p - p0) % DEPTH);
        mbar_expect_tx(bar, stage_bytes);
        tma_load_3d(bslot(p + 1), &mapB, bar, x0 - HX, y0 - 2, p + 1);
        if (!FIRST) tma_load_3d(aslot(p), &mapA, bar, x0 - HX, y0 - 1, p);
    };

    if (t == 0) {
        for (int q = 0; q <= DEPTH; ++q) mbar_init(bars + q, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    if (t == 0) {
        uint64_t* pro = bars + DEPTH;
        mbar_expect_tx(pro, 2 * BBYTES);
        tma_load_3d(bslot(p0 - 1), &mapB, pro, x0 - HX, y0 - 2, p0 - 1);
        tma_load_3d(bslot(p0), &mapB, pro, x0 - HX, y0 - 2, p0);
        for (int q = 0; q < DEPTH && p0 + q <= pend; ++q) issue_stage(p0 + q);
    }

    Dot2f dot, nrm;
    int issued_upto = min(p0 + DEPTH - 1, pend);
    for (int p = p0; p <= pend; ++p) {
        bool ok = true;
        if (p == p0) ok = mbar_wait(bars + DEPTH, 0);
        ok = ok && mbar_wait(bars + ((p - p0) % DEPTH), (unsigned)(((p - p0) / DEPTH) & 1));
        if (!ok) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;

        // ---- w on plane p over the tile + 1 halo ring
        const float* Bm = bslot(p - 1);
        const float* Bc = bslot(p);
        const float* Bp = bslot(p + 1);
        const float* Ac = aslot(p);
        float* Wp = wslot(p);
        const bool pin = p >= 0 && p < g.nz;
        for (int e = t; e < WW * WH; e += FNT) {
            const int c = e % WW, r = e / WW;
            const int x = x0 - 1 + c, y = y0 - 1 + r;
            float w = 0.f;
            if (pin && x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
                const int bi = (r + 1) * BW + (c + HX - 1);
                w = ax * (Bc[bi - 1] + Bc[bi + 1]) + ay * (Bc[bi - BW] + Bc[bi + BW]) + az * (Bm[bi] + Bp[bi]) +
                    bc * Bc[bi];
                if (!FIRST) w += ba * Ac[r * BW + (c + HX - 1)];
            }
            Wp[e] = w;
        }
        __syncthreads();

        // ---- finish the interior of plane q = p - 1
        const int q = p - 1;
        if (q >= z0) {
            const float* Wm = wslot(q - 1);
            const float* Wc = wslot(q);
            const float* Wn = wslot(q + 1);
            const int i4 = (t & 31) * 4;
            for (int k = t >> 5; k < FTY; k += FNT / 32) {
                const int y = y0 + k;
                const int x = x0 + i4;
                if (y >= g.ny || x >= g.nx) continue;
                float wv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int wi = (k + 1) * WW + (i4 + u + 1);
                    const float w = Wc[wi];
                    const float aw = kx * (Wc[wi - 1] + Wc[wi + 1]) + ky * (Wc[wi - WW] + Wc[wi + WW]) +
                                     kz * (Wm[wi] + Wn[wi]) + kc * w;
                    dot.add_prod(w, aw);
                    nrm.add_prod(w, w);
                    wv[u] = w;
                }
                float* dst = a.W + ((int64_t)q * g.ny + y) * g.nx + x;
                *reinterpret_cast<float4*>(dst) = make_float4(wv[0], wv[1], wv[2], wv[3]);
            }
        }
        __syncthreads();
        // ---- refill: B plane p-1's slot and A plane p's slot are free now
        if (t == 0 && p + DEPTH <= pend) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_stage(p + DEPTH);
            issued_upto = p + DEPTH;
        }
    }
    if (abort_flag) {
        // drain this CTA's copies (bounded) before leaving; report the timeout
        if (t == 0) {
            atomicOr(&a.st->status, 1);
            mbar_wait(bars + DEPTH, 0);
            for (int q = 0; q < DEPTH; ++q) mbar_wait(bars + q, 0), mbar_wait(bars + q, 1);
        }
        __syncthreads();
        return;
    }
    (void)issued_upto;

    // ---- deterministic grid reduction of (w.w, w.Aw)
    const double d_nrm = block_sum<FNT>(nrm.value(), shred);
    const double d_dot = block_sum<FNT>(dot.value(), shred);
    const int64_t nb = (int64_t)gridDim.x * gridDim.y * gridDim.z;
    const int64_t slot = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (t == 0) a.red.partials[nb + slot] = d_dot;
    if (!grid_arrive(d_nrm, a.red.partials, a.red.counter, slot, nb, &flag)) return;
    const double nw2 = grid_finish<FNT>(a.red.partials, nb, a.red.counter, shred);
    const double wAw = grid_finish<FNT>(a.red.partials + nb, nb, a.red.counter, shred);
    __shared__ double snext;
    __shared__ int cont;
    if (t == 0) {
        const int j = a.j, m = a.m;
        const double beta = sqrt(nw2);
        a.H[(int64_t)(j + 1) * m + j] = beta;
        const double bj = FIRST ? 0.0 : a.H[(int64_t)j * m + (j - 1)];
        const double nav = sqrt(alpha * alpha + bj * bj + beta * beta);  // ||A v_j||
        if (!(beta > 1e-12 * nav) || !isfinite(beta)) {
            a.st->done = 1;
            a.st->m_used = j + 1;
            cont = 0;
        } else {
            a.st->s[j + 1] = 1.0 / beta;
            snext = 1.0 / beta;
            if (j + 1 < m) {
                a.H[(int64_t)j * m + (j + 1)] = beta;
                a.H[(int64_t)(j + 1) * m + (j + 1)] = wAw / nw2;  // alpha_{j+1}
            }
            cont = (j + 1 < m) ? 1 : 0;
        }
    }
    __syncthreads();
    if (!cont) return;
    for (int r = 0; r < a.cd.o; ++r) {
        double v = 0.0;
        for (int64_t e = a.cd.rp[r] + t; e < a.cd.rp[r + 1]; e += FNT)
            v += a.cd.val[e] * (double)__ldcg(a.W + a.cd.col[e]);
        v = block_sum<FNT>(v, shred);
        if (t == 0) a.P[(int64_t)r * a.m + (a.j + 1)] = snext * v;
    }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*PfnEncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PfnEncodeTiled encode_fn() {
    static PfnEncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PfnEncodeTiled)p;
    }
    return fn;
}

// Whether the single-pass TMA iteration applies: FP32 grid, rows a multiple
// of 16 bytes (TMA stride rule), extents within TMA limits.
bool fused_tma_supported(const Prob* p) {
    const Sys* s = p->sys;
    if (s->kind != 0 || p->prec != KV_FP32) return false;
    const int64_t nx = s->dims[0], ny = s->ndim >= 2 ? s->dims[1] : 1, nz = s->ndim >= 3 ? s->dims[2] : 1;
    if (nx % 4 != 0 || nx > ((int64_t)1 << 31) || ny > ((int64_t)1 << 31) || nz > ((int64_t)1 << 31)) return false;
    return encode_fn() != nullptr;
}

static int make_map(CUtensorMap* m, void* base, const Sys* s, int box_h) {
    const int64_t nx = s->dims[0], ny = s->ndim >= 2 ? s->dims[1] : 1, nz = s->ndim >= 3 ? s->dims[2] : 1;
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)BW, (cuuint32_t)box_h, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return KV_ECUDA;
    }
    return KV_OK;
}

int fused_tma_blocks(const Prob* p, int* zc_out) {
    const Sys* s = p->sys;
    const int64_t nx = s->dims[0], ny = s->ndim >= 2 ? s->dims[1] : 1, nz = s->ndim >= 3 ? s->dims[2] : 1;
    const int64_t bx = (nx + FTX - 1) / FTX, by = (ny + FTY - 1) / FTY;
    // z chunk: about 12 waves of 2 resident CTAs per SM, at least 16 planes
    const int64_t target = 152LL * 2 * 12;
    int64_t nzc = (target + bx * by - 1) / (bx * by);
    if (nzc < 1) nzc = 1;
    int64_t zc = (nz + nzc - 1) / nzc;
    if (zc < 16) zc = 16;
    if (zc > nz) zc = nz;
    *zc_out = (int)zc;
    return (int)(bx * by * ((nz + zc - 1) / zc));
}

int launch_lanczos_fused(Prob* p, int j, int it, const void* B, const void* A, void* Wout) {
    const Sys* s = p->sys;
    StencilGeom g;
    g.nx = s->dims[0];
    g.ny = s->ndim >= 2 ? s->dims[1] : 1;
    g.nz = s->ndim >= 3 ? s->dims[2] : 1;
    g.kx = s->coef / (s->h[0] * s->h[0]);
    g.ky = s->ndim >= 2 ? s->coef / (s->h[1] * s->h[1]) : 0.0;
    g.kz = s->ndim >= 3 ? s->coef / (s->h[2] * s->h[2]) : 0.0;
    g.kc = -2.0 * (g.kx + g.ky + g.kz);
    CUtensorMap mB, mA;
    int rc = make_map(&mB, const_cast<void*>(B), s, BH);
    if (!rc) rc = make_map(&mA, const_cast<void*>(A), s, AH);
    if (rc) return rc;
    int zc;
    fused_tma_blocks(p, &zc);
    dim3 grd((unsigned)((g.nx + FTX - 1) / FTX), (unsigned)((g.ny + FTY - 1) / FTY), (unsigned)((g.nz + zc - 1) / zc));
    FusedArgs a;
    a.W = (float*)Wout;
    a.g = g;
    a.zc = zc;
    a.st = p->d_state + j;
    a.H = p->d_H + (int64_t)j * (p->m + 1) * p->m;
    a.P = p->d_P + (int64_t)j * p->o * p->m;
    a.cd = CDesc{p->o, p->d_crp, p->d_ccol, p->d_cval};
    a.m = p->m;
    a.j = it;
    a.red = p->red;
    static bool attr_set = false;
    if (!attr_set) {
        KV_CHECK_CUDA(cudaFuncSetAttribute(k_lanczos_fused_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TOTAL));
        KV_CHECK_CUDA(cudaFuncSetAttribute(k_lanczos_fused_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TOTAL));
        attr_set = true;
    }
    LaunchScope ls(p->ctx, "lanczos_fused");
    if (it == 0)
        k_lanczos_fused_tma<true><<<grd, FNT, SMEM_TOTAL, p->ctx->stream>>>(mB, mA, a);
    else
        k_lanczos_fused_tma<false><<<grd, FNT, SMEM_TOTAL, p->ctx->stream>>>(mB, mA, a);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

}  // namespace kv
