// k_stencil.cu -- matrix-free grid Laplacian Lanczos passes (Alg. 3 / Alg. 4).
//
// A = coef * (discrete Laplacian, spacing h per axis) with a coefficient per
// grid face (Dirichlet-0 unless the system says otherwise).  One
// Lanczos iteration j runs as two passes over the grid:
//   alpha pass:  alpha_j = v_j . A v_j                         (reads v_j)
//   update pass: w = A v_j - alpha_j v_j - beta_j v_{j-1}, stored over v_{j-1};
//                beta_{j+1} = ||w||; P[:, j+1] = C w / beta_{j+1} (reads v_j,
//                v_{j-1}, writes w)
// Alg. 3 takes alpha_j = v_j . (A v_j - beta_j v_{j-1}); the two agree in
// exact arithmetic because v_j is orthogonal to v_{j-1}.  Vectors are stored
// unnormalised and scaled by s[j] = 1 / beta_j on read, so only two n-vectors
// are live.  All scalars stay on the device; each pass's last block finishes
// the reduction and writes them, so no host round trip happens per iteration.
//
// Threads own an (x, y) column of the grid and march over a chunk of z planes,
// keeping the z-1 / z / z+1 values in registers; the x and y neighbours are
// re-read through L1.  The FP32 form stores vectors in float, computes A v in
// float and accumulates every dot product error-free (Dot2) before the double
// block reduction.
#include <type_traits>

#include "kv_internal.h"
#include "reduce.cuh"

namespace kv {

constexpr int SBX = 32, SBY = 8, SNT = SBX * SBY;

int stencil_blocks(const StencilGeom& g, int* zc_out) {
    const int64_t bx = (g.nx + SBX - 1) / SBX, by = (g.ny + SBY - 1) / SBY;
    // z chunk: enough blocks for ~16 waves of 8 resident blocks on 152 SMs,
    // chunks of at least 8 planes so the float accumulators see long runs.
    const int64_t target = 152LL * 8 * 16;
    int64_t nzc = (target + bx * by - 1) / (bx * by);
    if (nzc < 1) nzc = 1;
    int64_t zc = (g.nz + nzc - 1) / nzc;
    if (zc < 8) zc = 8;
    if (zc > g.nz) zc = g.nz;
    *zc_out = (int)zc;
    const int64_t bz = (g.nz + zc - 1) / zc;
    return (int)(bx * by * bz);
}

static StencilGeom geom_of(const Sys* s) {
    StencilGeom g;
    g.nx = s->dims[0];
    g.ny = s->ndim >= 2 ? s->dims[1] : 1;
    g.nz = s->ndim >= 3 ? s->dims[2] : 1;
    g.kx = s->coef / (s->h[0] * s->h[0]);
    g.ky = s->ndim >= 2 ? s->coef / (s->h[1] * s->h[1]) : 0.0;
    g.kz = s->ndim >= 3 ? s->coef / (s->h[2] * s->h[2]) : 0.0;
    g.kc = -2.0 * (g.kx + g.ky + g.kz);
    const double kap[3] = {g.kx, g.ky, g.kz};
    for (int f = 0; f < 6; ++f) g.rho[f] = kap[f >> 1] > 0.0 ? s->face[f] / kap[f >> 1] : 0.0;
    return g;
}

// gather of C x for row r by the whole (last) block; result in thread 0
template <typename T>
__device__ double c_gather_row(const CDesc& cd, int r, const T* x, double* sh, int* status) {
    double v = 0.0;
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    for (int64_t e = cd.rp[r] + t; e < cd.rp[r + 1]; e += SNT) v += c_entry(cd, e, x, status);
    return block_sum<SNT>(v, sh);
}

// ------------------------------------------------------------------ init --
template <typename T>
__global__ void __launch_bounds__(SNT) k_stencil_init_box(T* __restrict__ B, StencilGeom g, int zc,
                                                          int64_t lx, int64_t ly, int64_t lz, int64_t hx,
                                                          int64_t hy, int64_t hz, double value,
                                                          ColState* st, double* H0, double* P, CDesc cd, int m,
                                                          Reduce red) {
    __shared__ double sh[SNT / 32];
    __shared__ int flag;
    const int64_t x = (int64_t)blockIdx.x * SBX + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * SBY + threadIdx.y;
    const int64_t z0 = (int64_t)blockIdx.z * zc;
    const int64_t z1 = min(z0 + zc, g.nz);
    const T tv = (T)value;
    double acc = 0.0;
    if (x < g.nx && y < g.ny) {
        const bool inxy = x >= lx && x < hx && y >= ly && y < hy;
        int64_t idx = (z0 * g.ny + y) * g.nx + x;
        const int64_t P2 = g.nx * g.ny;
        int64_t cnt = 0;
        for (int64_t z = z0; z < z1; ++z, idx += P2) {
            const bool in = inxy && z >= lz && z < hz;
            B[idx] = in ? tv : (T)0;
            cnt += in ? 1 : 0;
        }
        acc = (double)cnt * (double)tv * (double)tv;
    }
    const double part = block_sum<SNT>(acc, sh);
    const int64_t slot = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int64_t nb = (int64_t)gridDim.x * gridDim.y * gridDim.z;
    if (!grid_arrive(part, red.partials, red.counter, slot, nb, &flag)) return;
    const double tot = grid_finish<SNT>(red.partials, nb, red.counter, sh);
    __shared__ double s0;
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    if (t == 0) {
        const double b0 = sqrt(tot);
        st->beta0 = b0;
        st->m_used = m;
        st->status = 0;
        if (!(b0 > 0.0) || !isfinite(b0)) {
            st->done = 1;
            st->m_used = 0;
            s0 = 0.0;
        } else {
            st->done = 0;
            st->s[0] = 1.0 / b0;
            s0 = 1.0 / b0;
            // alpha_0 = v_0 . A v_0 for the box indicator in closed form: by
            // summation by parts v . A v = -sum_a kappa_a sum_edges (difference)^2,
            // and the indicator differs across exactly the two faces of the box
            // on each axis (towards the zero ghost where the box meets the
            // grid boundary), one edge per face cell.
            // A face of the box on a face of the grid couples to the ghost
            // with gamma = rho kappa instead of kappa.
            const double ex = (double)(hx - lx), ey = (double)(hy - ly), ez = (double)(hz - lz);
            const double wx = g.kx * ((lx > 0 ? 1.0 : g.rho[0]) + (hx < g.nx ? 1.0 : g.rho[1]));
            const double wy = g.ky * ((ly > 0 ? 1.0 : g.rho[2]) + (hy < g.ny ? 1.0 : g.rho[3]));
            const double wz = g.kz * ((lz > 0 ? 1.0 : g.rho[4]) + (hz < g.nz ? 1.0 : g.rho[5]));
            H0[0] = -(wx * ey * ez + wy * ex * ez + wz * ex * ey) / (ex * ey * ez);
        }
    }
    __syncthreads();
    if (cd.o > PROJ_INLINE_MAX) return;  // launch_project takes the rows
    for (int r = 0; r < cd.o; ++r) {
        const double v = c_gather_row<T>(cd, r, B, sh, &st->status);
        if (t == 0) P[(int64_t)r * m + 0] = s0 * v;
    }
}

// ----------------------------------------------------------------- alpha --
template <typename T>
__global__ void __launch_bounds__(SNT) k_stencil_alpha(const T* __restrict__ B, StencilGeom g, int zc,
                                                       ColState* st, double* H, int m, int j, Reduce red) {
    if (st->done) return;
    __shared__ double sh[SNT / 32];
    __shared__ int flag;
    const int64_t x = (int64_t)blockIdx.x * SBX + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * SBY + threadIdx.y;
    const int64_t z0 = (int64_t)blockIdx.z * zc;
    const int64_t z1 = min(z0 + zc, g.nz);
    typename AccOf<T>::type acc;
    if (x < g.nx && y < g.ny) {
        const T kx = (T)g.kx, ky = (T)g.ky, kz = (T)g.kz, kc = (T)g.kc;
        const int64_t P2 = g.nx * g.ny;
        int64_t idx = (z0 * g.ny + y) * g.nx + x;
        T cm = z0 > 0 ? B[idx - P2] : (T)0;
        T c = B[idx];
        const bool hl = x > 0, hr = x < g.nx - 1, hd = y > 0, hu = y < g.ny - 1;
        for (int64_t z = z0; z < z1; ++z, idx += P2) {
            const bool hm = z > 0, hp = z + 1 < g.nz;
            const T cp = hp ? B[idx + P2] : (T)0;
            T av;
            if constexpr (std::is_same<T, float>::value) {
                // difference form: neighbour - centre is exact for nearby values;
                // a face keeps the share rho of the ghost coupling (-rho c)
                const float dl = hl ? B[idx - 1] - c : -(float)g.rho[0] * c;
                const float dr = hr ? B[idx + 1] - c : -(float)g.rho[1] * c;
                const float dd = hd ? B[idx - g.nx] - c : -(float)g.rho[2] * c;
                const float du = hu ? B[idx + g.nx] - c : -(float)g.rho[3] * c;
                const float dm = hm ? cm - c : -(float)g.rho[4] * c;
                const float dp = hp ? cp - c : -(float)g.rho[5] * c;
                av = kx * (dl + dr) + ky * (dd + du) + kz * (dm + dp);
            } else {
                // pair-sum form: a face's ghost value is (1 - rho) c (0: Dirichlet)
                const T l = hl ? B[idx - 1] : (T)(1.0 - g.rho[0]) * c;
                const T r = hr ? B[idx + 1] : (T)(1.0 - g.rho[1]) * c;
                const T d = hd ? B[idx - g.nx] : (T)(1.0 - g.rho[2]) * c;
                const T u = hu ? B[idx + g.nx] : (T)(1.0 - g.rho[3]) * c;
                const T mz = hm ? cm : (T)(1.0 - g.rho[4]) * c;
                const T pz = hp ? cp : (T)(1.0 - g.rho[5]) * c;
                av = kx * (l + r) + ky * (d + u) + kz * (mz + pz) + kc * c;
            }
            acc.add_prod(c, av);
            cm = c;
            c = cp;
        }
    }
    const double part = block_sum<SNT>(acc.value(), sh);
    const int64_t slot = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int64_t nb = (int64_t)gridDim.x * gridDim.y * gridDim.z;
    if (!grid_arrive(part, red.partials, red.counter, slot, nb, &flag)) return;
    const double tot = grid_finish<SNT>(red.partials, nb, red.counter, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const double s = st->s[j];
        H[(int64_t)j * m + j] = s * s * tot;  // alpha_j
        if (!isfinite(tot)) {
            st->status |= KV_ST_NONFINITE;
            st->done = 1;
            st->m_used = j;
        }
    }
}

// ---------------------------------------------------------------- update --
template <typename T, bool FIRST>
__global__ void __launch_bounds__(SNT) k_stencil_update(const T* __restrict__ B, T* __restrict__ A,
                                                        StencilGeom g, int zc, ColState* st, double* H,
                                                        double* P, CDesc cd, int m, int j, Reduce red) {
    if (st->done) return;
    __shared__ double sh[SNT / 32];
    __shared__ int flag;
    const double sj = st->s[j];
    const double alpha = H[(int64_t)j * m + j];
    const double c1 = sj;
    const double c2 = sj * (g.kc - alpha);
    const double c3 = FIRST ? 0.0 : -H[(int64_t)j * m + (j - 1)] * st->s[j - 1];
    const int64_t x = (int64_t)blockIdx.x * SBX + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * SBY + threadIdx.y;
    const int64_t z0 = (int64_t)blockIdx.z * zc;
    const int64_t z1 = min(z0 + zc, g.nz);
    typename AccOf<T>::type acc;
    if (x < g.nx && y < g.ny) {
        const T ax = (T)(c1 * g.kx), ay = (T)(c1 * g.ky), az = (T)(c1 * g.kz);
        const T bc = (T)c2, ba = (T)c3;
        // float form: w = sum_a (s kappa_a) L_a + (-alpha s) c + (-beta s') a with
        // L_a the difference-form second difference and every coefficient split
        // into a float pair (hi + lo), accumulated as one FMA chain
        const CoefPair fx = split_coef(c1 * g.kx), fy = split_coef(c1 * g.ky), fz = split_coef(c1 * g.kz);
        const CoefPair fc = split_coef(-alpha * sj), fa = split_coef(c3);
        const int64_t P2 = g.nx * g.ny;
        int64_t idx = (z0 * g.ny + y) * g.nx + x;
        T cm = z0 > 0 ? B[idx - P2] : (T)0;
        T c = B[idx];
        const bool hl = x > 0, hr = x < g.nx - 1, hd = y > 0, hu = y < g.ny - 1;
        for (int64_t z = z0; z < z1; ++z, idx += P2) {
            const bool hm = z > 0, hp = z + 1 < g.nz;
            const T cp = hp ? B[idx + P2] : (T)0;
            T w;
            if constexpr (std::is_same<T, float>::value) {
                // difference form; a face keeps the share rho of the ghost coupling
                const float dl = hl ? B[idx - 1] - c : -(float)g.rho[0] * c;
                const float dr = hr ? B[idx + 1] - c : -(float)g.rho[1] * c;
                const float dd = hd ? B[idx - g.nx] - c : -(float)g.rho[2] * c;
                const float du = hu ? B[idx + g.nx] - c : -(float)g.rho[3] * c;
                const float dm = hm ? cm - c : -(float)g.rho[4] * c;
                const float dp = hp ? cp - c : -(float)g.rho[5] * c;
                const float Lx = dl + dr, Ly = dd + du, Lz = dm + dp;
                float acc2 = fx.lo * Lx;
                acc2 = fmaf(fy.lo, Ly, acc2);
                acc2 = fmaf(fz.lo, Lz, acc2);
                acc2 = fmaf(fc.lo, c, acc2);
                if (!FIRST) acc2 = fmaf(fa.lo, A[idx], acc2);
                acc2 = fmaf(fx.hi, Lx, acc2);
                acc2 = fmaf(fy.hi, Ly, acc2);
                acc2 = fmaf(fz.hi, Lz, acc2);
                acc2 = fmaf(fc.hi, c, acc2);
                if (!FIRST) acc2 = fmaf(fa.hi, A[idx], acc2);
                w = acc2;
            } else {
                // pair-sum form: a face's ghost value is (1 - rho) c (0: Dirichlet)
                const T l = hl ? B[idx - 1] : (T)(1.0 - g.rho[0]) * c;
                const T r = hr ? B[idx + 1] : (T)(1.0 - g.rho[1]) * c;
                const T d = hd ? B[idx - g.nx] : (T)(1.0 - g.rho[2]) * c;
                const T u = hu ? B[idx + g.nx] : (T)(1.0 - g.rho[3]) * c;
                const T mz = hm ? cm : (T)(1.0 - g.rho[4]) * c;
                const T pz = hp ? cp : (T)(1.0 - g.rho[5]) * c;
                w = ax * (l + r) + ay * (d + u) + az * (mz + pz) + bc * c;
                if (!FIRST) w += ba * A[idx];
            }
            A[idx] = w;
            acc.add_prod(w, w);
            cm = c;
            c = cp;
        }
    }
    const double part = block_sum<SNT>(acc.value(), sh);
    const int64_t slot = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int64_t nb = (int64_t)gridDim.x * gridDim.y * gridDim.z;
    if (!grid_arrive(part, red.partials, red.counter, slot, nb, &flag)) return;
    const double tot = grid_finish<SNT>(red.partials, nb, red.counter, sh);
    __shared__ double snext;
    __shared__ int cont;
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    if (t == 0) {
        const double beta = sqrt(tot);
        H[(int64_t)(j + 1) * m + j] = beta;
        const double bj = FIRST ? 0.0 : H[(int64_t)j * m + (j - 1)];
        const double nav = sqrt(alpha * alpha + bj * bj + beta * beta);  // ||A v_j||
        if (!(beta > 1e-12 * nav) || !isfinite(beta)) {
            if (!isfinite(beta)) st->status |= KV_ST_NONFINITE;
            st->done = 1;
            st->m_used = j + 1;
            cont = 0;
        } else {
            if (j + 1 < m) H[(int64_t)j * m + (j + 1)] = beta;
            st->s[j + 1] = 1.0 / beta;
            snext = 1.0 / beta;
            cont = (j + 1 < m) ? 1 : 0;
        }
    }
    __syncthreads();
    if (!cont || cd.o > PROJ_INLINE_MAX) return;
    for (int r = 0; r < cd.o; ++r) {
        const double v = c_gather_row<T>(cd, r, A, sh, &st->status);
        if (t == 0) P[(int64_t)r * m + (j + 1)] = snext * v;
    }
}

// --------------------------------------------------------------- launchers
static CDesc cdesc(const Prob* p) { return CDesc{p->o, p->d_crp, p->d_ccol, p->d_cval, p->N}; }

int launch_stencil_init_box(Prob* p, int j, void* B) {
    const StencilGeom g = geom_of(p->sys);
    int zc;
    stencil_blocks(g, &zc);
    dim3 blk(SBX, SBY), grd((unsigned)((g.nx + SBX - 1) / SBX), (unsigned)((g.ny + SBY - 1) / SBY),
                           (unsigned)((g.nz + zc - 1) / zc));
    const kv_column& c = p->cols[j];
    {
    LaunchScope ls(p->ctx, "stencil_init");
    const int64_t hz = p->sys->ndim >= 3 ? c.box_hi[2] : 1, lz = p->sys->ndim >= 3 ? c.box_lo[2] : 0;
    const int64_t hy = p->sys->ndim >= 2 ? c.box_hi[1] : 1, ly = p->sys->ndim >= 2 ? c.box_lo[1] : 0;
    ColState* st = p->d_state + j;
    double* H0 = p->d_H + (int64_t)j * (p->m + 1) * p->m;
    double* P = p->d_P + (int64_t)j * p->o * p->m;
    if (p->prec == KV_FP32)
        k_stencil_init_box<float><<<grd, blk, 0, p->ctx->stream>>>(
            (float*)B, g, zc, c.box_lo[0], ly, lz, c.box_hi[0], hy, hz, c.value, st, H0, P, cdesc(p), p->m, p->red);
    else
        k_stencil_init_box<double><<<grd, blk, 0, p->ctx->stream>>>(
            (double*)B, g, zc, c.box_lo[0], ly, lz, c.box_hi[0], hy, hz, c.value, st, H0, P, cdesc(p), p->m, p->red);
    KV_CHECK_CUDA(cudaGetLastError());
    }
    return launch_project(p, j, 1, B, 0, 0);
}

int launch_stencil_alpha(Prob* p, int j, int it, const void* B) {
    const StencilGeom g = geom_of(p->sys);
    int zc;
    stencil_blocks(g, &zc);
    dim3 blk(SBX, SBY), grd((unsigned)((g.nx + SBX - 1) / SBX), (unsigned)((g.ny + SBY - 1) / SBY),
                           (unsigned)((g.nz + zc - 1) / zc));
    LaunchScope ls(p->ctx, "stencil_alpha");
    ColState* st = p->d_state + j;
    double* H = p->d_H + (int64_t)j * (p->m + 1) * p->m;
    if (p->prec == KV_FP32)
        k_stencil_alpha<float><<<grd, blk, 0, p->ctx->stream>>>((const float*)B, g, zc, st, H, p->m, it, p->red);
    else
        k_stencil_alpha<double><<<grd, blk, 0, p->ctx->stream>>>((const double*)B, g, zc, st, H, p->m, it, p->red);
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

int launch_stencil_update(Prob* p, int j, int it, const void* B, void* A) {
    const StencilGeom g = geom_of(p->sys);
    int zc;
    stencil_blocks(g, &zc);
    dim3 blk(SBX, SBY), grd((unsigned)((g.nx + SBX - 1) / SBX), (unsigned)((g.ny + SBY - 1) / SBY),
                           (unsigned)((g.nz + zc - 1) / zc));
    LaunchScope ls(p->ctx, "stencil_update");
    ColState* st = p->d_state + j;
    double* H = p->d_H + (int64_t)j * (p->m + 1) * p->m;
    double* P = p->d_P + (int64_t)j * p->o * p->m;
    cudaStream_t s = p->ctx->stream;
    if (p->prec == KV_FP32) {
        if (it == 0)
            k_stencil_update<float, true><<<grd, blk, 0, s>>>((const float*)B, (float*)A, g, zc, st, H, P, cdesc(p), p->m, it, p->red);
        else
            k_stencil_update<float, false><<<grd, blk, 0, s>>>((const float*)B, (float*)A, g, zc, st, H, P, cdesc(p), p->m, it, p->red);
    } else {
        if (it == 0)
            k_stencil_update<double, true><<<grd, blk, 0, s>>>((const double*)B, (double*)A, g, zc, st, H, P, cdesc(p), p->m, it, p->red);
        else
            k_stencil_update<double, false><<<grd, blk, 0, s>>>((const double*)B, (double*)A, g, zc, st, H, P, cdesc(p), p->m, it, p->red);
    }
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

}  // namespace kv
