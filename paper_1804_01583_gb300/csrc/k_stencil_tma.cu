// k_stencil_tma.cu -- single-pass Lanczos iteration on the grid Laplacian
// (FP32 storage), with TMA-staged planes.
//
// One launch performs iteration j of the projected Lanczos loop (Alg. 3 with
// the Alg. 4 projection):
//     w = A v_j - alpha_j v_j - beta_j v_{j-1}           (written to a third buffer)
//     beta_{j+1}^2 = w . w,  alpha_{j+1} = (w . A w) / (w . w)
//     P[:, j+1] = C w / beta_{j+1}
// so alpha of the next iteration comes out of the same pass, and every
// iteration reads v_j and v_{j-1} once and writes w once: 12 bytes per grid
// point in FP32, the algorithmic minimum of a three-vector Lanczos step.
//
// w . A w without the neighbours of w on every side: for the Dirichlet-0
// Laplacian, summation by parts gives
//     w . A w = - sum_a kappa_a [ sum_p (w_p - w_{p - e_a})^2 + sum_{p on the
//               high face of axis a} w_p^2 ]            (w = 0 outside the grid)
// so each grid point only needs its backward neighbours, and every term has
// the same sign (no cancellation).
//
// Tiling: a CTA owns 124 (x) x 15 (y) points and marches over a chunk of z
// planes.  w is evaluated on the tile plus a one-point halo on the low x and
// y sides (a 128 x 16 region: warp k owns rows 2k and 2k+1, lane l the four
// consecutive x 4l..4l+3).  Per plane one elected thread issues TMA tile loads
// (cp.async.bulk.tensor, completion counted on an mbarrier) of v_j (x0-4 ..
// x0+123 with 2 rows of halo below and 1 above, plus a 4-column side box for
// the x0+124 neighbour) and v_{j-1} into a shared-memory ring four planes
// ahead of the compute (two CTAs per SM, so eight stages, about 140 KB, in
// flight per SM); TMA fills coordinates outside the grid with zeros, which is
// the Dirichlet-0 boundary.  A grid face with its own coefficient gamma
// (insulated, heat exchange) replaces the difference to that zero ghost by
// -(gamma / kappa) c, and its edge term in w . A w by gamma w^2.  Box rows are 512 bytes, so every float4 row load
// is conflict-free; the x neighbours of a thread's four points come from the
// adjacent lanes (shuffles).  The x-1 neighbour of w comes from the next lane
// (shuffle), y-1 from the warp's own other row or the shared w plane, z-1
// from registers kept from the previous plane.  w goes to a buffer no CTA
// reads in this pass, so tiles never race on halos.
//
// The update is evaluated in float with the difference form of the Laplacian
// ((l - c) + (r - c): exact subtraction for nearby values) and one FMA chain
// with the double coefficients rounded to float; both dot
// products are summed per plane in float (squared differences per axis,
// weighted once per plane), accumulated over the planes as TwoSum float
// pairs and reduced across threads and CTAs in double.
//
// Every mbarrier wait is bounded; on expiry the CTA sets the column's status
// word (reported as KV_ETIMEOUT), drains its outstanding copies with bounded
// waits and leaves.
#include <cuda.h>

#include <type_traits>

#include "kv_internal.h"
#include "reduce.cuh"
#include "tma.cuh"

namespace kv {

constexpr int FNT = 256;
constexpr int TXI = 124, TYI = 15;      // interior points of a tile
constexpr int WC = 128, WR = 16;        // w region: x0-4 .. x0+123, y0-1 .. y0+14
constexpr int BBW = 128, BBH = 18;      // v_j box: x0-4 .. x0+123, y0-2 .. y0+15 (512-byte rows)
constexpr int SBW = 4, SBH = 18;        // v_j side box: x0+124 .. x0+127, same rows
constexpr int ABW = 128, ABH = 16;      // v_{j-1} box: x0-4 .. x0+123, y0-1 .. y0+14
constexpr int DEPTH = 4;                // stages in flight (x 2 CTAs per SM)
constexpr int RB = DEPTH + 2, RA = DEPTH;
constexpr int BBYTES = BBW * BBH * 4;   // 9216
constexpr int SBYTES = SBW * SBH * 4;   // 288
constexpr int ABYTES = ABW * ABH * 4;   // 8192
constexpr int BSTRIDE = BBYTES;
constexpr int SSTRIDE = (SBYTES + 127) / 128 * 128;
constexpr int ASTRIDE = ABYTES;
constexpr int WSTRIDE = WC * WR * 4;
constexpr int SMEM_MAIN = RB * BSTRIDE + RB * SSTRIDE + RA * ASTRIDE + 2 * WSTRIDE;
constexpr int SMEM_TOTAL = SMEM_MAIN + 128 + 1024;  // + barriers + alignment slack
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
    // 1-D grid of z chunks, each nbx * nby full-width tiles then nby_s
    // narrow ones
    int nbx, nby;
    int sg_log2, nby_s;  // narrow tiles: 2^sg_log2 lanes per row pair; 0 = none
    // grid faces (x low, x high, y low, y high, z low, z high), used when the
    // system's boundary is not Dirichlet-0: rho = gamma / kappa, the share of
    // the ghost coupling a face keeps, and gamma itself (the face term of w . A w)
    float rho[6], gam[6];
};

// One CTA's tile and chunk of z planes.  LG = log2 of the lanes that share
// a row pair: 5 for a full-width tile (32 lanes over 128 columns, one warp
// per 2 rows); 2, 3 or 4 for a narrow tile of the last x columns (G = 4, 8 or
// 16 lanes over 4G columns, one warp per 2 * 32/G rows).  Both shapes cover
// a 2048-point w region and use the same shared-memory slots; the shape is a
// compile-time constant, so the box offsets fold into the load instructions.
// Returns false when a stage wait expired (the copies are drained and the
// timeout reported); otherwise this thread's sums of w.w and -w.Aw.
template <bool FIRST, int LG, bool FACES>
__device__ __forceinline__ bool fused_tile(const CUtensorMap* mB, const CUtensorMap* mS, const CUtensorMap* mA,
                                           const FusedArgs& a, int tx, int ty, int tz, unsigned char* sm,
                                           int& abort_flag, double& sum_n, double& sum_e) {
    constexpr bool NARROW = LG < 5;
    constexpr int G = 1 << LG;         // lanes per row pair
    constexpr int RGW = 32 >> LG;      // row pairs per warp
    constexpr int WCM = 4 * G;         // columns of the w region and of both boxes
    constexpr int WRM = 16 * RGW;      // rows of the w region
    float* sB = (float*)sm;
    float* sS = (float*)(sm + RB * BSTRIDE);
    float* sA = (float*)(sm + RB * (BSTRIDE + SSTRIDE));
    float* sW = (float*)(sm + RB * (BSTRIDE + SSTRIDE) + RA * ASTRIDE);
    uint64_t* bars = (uint64_t*)(sm + SMEM_MAIN);  // DEPTH stage barriers + 1 prologue barrier
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const StencilGeom& g = a.g;
    const int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz;
    const int x0 = tx * TXI, y0 = ty * (WRM - 1);
    const int z0 = tz * a.zc;
    constexpr unsigned bbytes = (unsigned)(WCM * (WRM + 2) * 4);
    const int z1 = min(z0 + a.zc, nz);
    const int p0 = z0 - 1;  // w planes p0 .. z1-1; the interior work runs for z0 .. z1-1

    const double sj = a.st->s[a.j];
    const double alpha = a.H[(int64_t)a.j * a.m + a.j];
    // the coefficients of w = s_j A v_j - alpha s_j v_j - beta s_{j-1} v_{j-1},
    // rounded to float once (with the difference form of the Laplacian this
    // is as accurate as carrying them as float pairs: the error is that of
    // the FP32 storage)
    const float fx = (float)(sj * g.kx), fy = (float)(sj * g.ky), fz = (float)(sj * g.kz);
    const float fc = (float)(-alpha * sj);
    const float fa = (float)(FIRST ? 0.0 : -a.H[(int64_t)a.j * a.m + (a.j - 1)] * a.st->s[a.j - 1]);
    const float kx = (float)g.kx, ky = (float)g.ky, kz = (float)g.kz;

    auto ring = [](int plane, int n) { return ((plane % n) + n) % n; };
    auto load_b = [&](int plane, uint64_t* bar) {  // v_j plane: main box + side box, same ring slot
        const int k = ring(plane, RB);
        tma_load_3d(sB + (size_t)k * (BSTRIDE / 4), mB, bar, x0 - 4, y0 - 2, plane);
        if (!NARROW) tma_load_3d(sS + (size_t)k * (SSTRIDE / 4), mS, bar, x0 + 124, y0 - 2, plane);
    };
    constexpr unsigned bplane_bytes = bbytes + (NARROW ? 0u : (unsigned)SBYTES);
    constexpr unsigned stage_bytes = bplane_bytes + (FIRST ? 0u : (unsigned)ABYTES);
    auto issue_stage = [&](int p) {  // B plane p+1, A plane p -> stage barrier of p
        uint64_t* bar = bars + ((p - p0) % DEPTH);
        mbar_expect_tx(bar, stage_bytes);
        load_b(p + 1, bar);
        if (!FIRST) tma_load_3d(sA + (size_t)ring(p, RA) * (ASTRIDE / 4), mA, bar, x0 - 4, y0 - 1, p);
    };

    // this thread's points: rows r0, r0 + 1; columns c = 4 cg + u
    const int cg = lane & (G - 1);
    const int r0 = 2 * (warp * RGW + (lane >> LG));
    const int xb = x0 - 4 + 4 * cg;                   // x of u = 0 (multiple of 4)
    const bool xin = xb >= 0 && xb < nx;              // nx % 4 == 0: all four or none
    const bool yin0 = (y0 - 1 + r0) >= 0 && (y0 - 1 + r0) < ny;
    const bool yin1 = (y0 + r0) < ny;                 // y0 + r0 >= 0 always
    const bool inner_x = cg >= 1 && xin;              // c >= 4: inside the tile
    const bool inner0 = inner_x && r0 >= 1 && yin0;   // row r0 interior (r0 >= 1)
    const bool inner1 = inner_x && yin1;              // row r0 + 1 >= 1 always
    const bool xhi3 = xin && (xb + 3 == nx - 1);      // u = 3 on the high x face
    const bool yhi0 = (y0 - 1 + r0) == ny - 1, yhi1 = (y0 + r0) == ny - 1;
    const bool ylo0 = (y0 - 1 + r0) == 0, ylo1 = (y0 + r0) == 0;
    const bool xlo0 = xb == 0;                        // u = 0 on the low x face

    if (t == 0) {
        for (int q = 0; q <= DEPTH; ++q) mbar_init(bars + q, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    int issued_upto = p0 - 1;
    if (t == 0) {
        uint64_t* pro = bars + DEPTH;
        mbar_expect_tx(pro, 2 * bplane_bytes);
        load_b(p0 - 1, pro);
        load_b(p0, pro);
        for (int q = 0; q < DEPTH && p0 + q <= z1 - 1; ++q) {
            issue_stage(p0 + q);
            issued_upto = p0 + q;
        }
    }

    float4 zp0 = make_float4(0.f, 0.f, 0.f, 0.f), zp1 = zp0;  // w of the previous plane
    float an_hi = 0.f, an_lo = 0.f, ae_hi = 0.f, ae_lo = 0.f;
    int pfail = -1;
    // ring positions of B(p-1), B(p), B(p+1), A(p) and the stage barrier /
    // parity of plane p, rotated by one per plane
    int sbm = (((p0 - 1) % RB) + RB) % RB, sbc = ((p0 % RB) + RB) % RB, sbp = (((p0 + 1) % RB) + RB) % RB;
    int sac = ((p0 % RA) + RA) % RA, sst = 0;
    unsigned sph = 0;
    // offset of this thread's row r0 in w at plane p (the row r0 + 1 is nx further)
    int64_t woff = ((int64_t)p0 * ny + (y0 - 1 + r0)) * nx + xb;
    const int64_t plane = (int64_t)nx * ny;
    for (int p = p0; p <= z1 - 1; ++p) {
        bool ok = true;
        if (p == p0) ok = mbar_wait(bars + DEPTH, 0);
        ok = ok && mbar_wait(bars + sst, sph);
        // No barrier here: each thread's own wait makes the stage visible to
        // it, and the w plane written below is the other half of a double
        // buffer whose last readers passed the previous plane's barrier.
        // A failed wait is acted on after the barrier below.
        if (!ok) abort_flag = 1;
        const float* Bm = sB + (size_t)sbm * (BSTRIDE / 4);
        const float* Bc = sB + (size_t)sbc * (BSTRIDE / 4);
        const float* Bp = sB + (size_t)sbp * (BSTRIDE / 4);
        const float* Sc = sS + (size_t)sbc * (SSTRIDE / 4);
        const float* Ac = sA + (size_t)sac * (ASTRIDE / 4);
        float* Wp = sW + (p & 1) * (WSTRIDE / 4);
        const bool pin = p >= 0 && p < nz;

        // ---- w on this thread's 2 x 4 points
        float4 w2[2];
        // v_j box rows r0 .. r0+3 (w rows r0-1 .. r0+2): the y neighbours and
        // centres of both of this thread's rows, each loaded once.  In
        // full-width tiles every box row is 512 bytes, so each float4 row
        // load is four conflict-free wavefronts.
        float4 brows[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) brows[q] = *reinterpret_cast<const float4*>(Bc + (r0 + q) * WCM + 4 * cg);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = r0 + h;
            const bool valid = pin && xin && (h == 0 ? yin0 : yin1);
            const int bo = (r + 1) * WCM + 4 * cg;
            const float4 c4 = brows[h + 1];
            // x neighbours from the adjacent lanes.  cg = 0's left value feeds
            // only w(x0-4), which nothing reads; the right one of cg = G-1 is
            // column x0+124 of the side box (full width) or lies beyond the
            // grid (a narrow tile covers the last columns): zero
            const float lft = __shfl_up_sync(0xffffffffu, c4.w, 1);
            float rgt = __shfl_down_sync(0xffffffffu, c4.x, 1);
            if (cg == G - 1) rgt = NARROW ? 0.f : Sc[(r + 1) * SBW];
            const float4 d4 = brows[h];
            const float4 u4 = brows[h + 2];
            const float4 m4 = *reinterpret_cast<const float4*>(Bm + bo);
            const float4 p4 = *reinterpret_cast<const float4*>(Bp + bo);
            float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!FIRST) a4 = *reinterpret_cast<const float4*>(Ac + r * WCM + 4 * cg);
            const float cc[4] = {c4.x, c4.y, c4.z, c4.w};
            const float xl[4] = {lft, c4.x, c4.y, c4.z};
            const float xr[4] = {c4.y, c4.z, c4.w, rgt};
            const float dd[4] = {d4.x, d4.y, d4.z, d4.w};
            const float uu[4] = {u4.x, u4.y, u4.z, u4.w};
            const float mm[4] = {m4.x, m4.y, m4.z, m4.w};
            const float pp[4] = {p4.x, p4.y, p4.z, p4.w};
            const float aa[4] = {a4.x, a4.y, a4.z, a4.w};
            float wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float c = cc[u];
                float Lx, Ly, Lz;
                if (!FACES) {
                    Lx = (xl[u] - c) + (xr[u] - c);
                    Ly = (dd[u] - c) + (uu[u] - c);
                    Lz = (mm[u] - c) + (pp[u] - c);
                } else {
                    // a face replaces the difference to the ghost by -rho c
                    const bool ylo = h == 0 ? ylo0 : ylo1, yhi = h == 0 ? yhi0 : yhi1;
                    const float dl = (u == 0 && xlo0) ? -a.rho[0] * c : xl[u] - c;
                    const float dr = (u == 3 && xhi3) ? -a.rho[1] * c : xr[u] - c;
                    const float dn = ylo ? -a.rho[2] * c : dd[u] - c;
                    const float dup = yhi ? -a.rho[3] * c : uu[u] - c;
                    const float dm = p == 0 ? -a.rho[4] * c : mm[u] - c;
                    const float dp = p == nz - 1 ? -a.rho[5] * c : pp[u] - c;
                    Lx = dl + dr;
                    Ly = dn + dup;
                    Lz = dm + dp;
                }
                float acc = fx * Lx;
                acc = fmaf(fy, Ly, acc);
                acc = fmaf(fz, Lz, acc);
                acc = fmaf(fc, c, acc);
                if (!FIRST) acc = fmaf(fa, aa[u], acc);
                wv[u] = valid ? acc : 0.f;
            }
            w2[h] = make_float4(wv[0], wv[1], wv[2], wv[3]);
            *reinterpret_cast<float4*>(Wp + r * WCM + 4 * cg) = w2[h];
        }
        __syncthreads();  // w of this plane visible; B(p-1) and A(p) no longer read
        if (abort_flag) {  // some thread's wait expired: the stage may be incomplete
            pfail = p;
            break;
        }
        if (t == 0 && p + DEPTH <= z1 - 1) {
            // stage p + DEPTH reuses this stage's barrier, B(p-1)'s slot (it takes
            // B(p + DEPTH + 1)) and A(p)'s slot
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int q = p + DEPTH;
            uint64_t* bar = bars + sst;
            mbar_expect_tx(bar, stage_bytes);
            load_b(q + 1, bar);  // lands in B(p-1)'s slot: (q + 1) - (p - 1) = RB
            if (!FIRST) tma_load_3d((void*)Ac, mA, bar, x0 - 4, y0 - 1, q);
            issued_upto = q;
        }

        // ---- interior of plane p: norm, edge terms of w . A w, store
        if (p >= z0) {
            const float left0 = __shfl_up_sync(0xffffffffu, w2[0].w, 1);
            const float left1 = __shfl_up_sync(0xffffffffu, w2[1].w, 1);
            float4 up0 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r0 >= 1) up0 = *reinterpret_cast<const float4*>(Wp + (r0 - 1) * WCM + 4 * cg);
            // squared backward differences per axis, weighted once per plane
            float tx = 0.f, ty = 0.f, tz = 0.f, tn = 0.f, tg = 0.f;
            const bool zhi = p == nz - 1;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool inn = h == 0 ? inner0 : inner1;
                if (!inn) continue;
                const float4 w4 = w2[h];
                const float4 up = h == 0 ? up0 : w2[0];
                const float4 zp = h == 0 ? zp0 : zp1;
                const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
                const float lf[4] = {h == 0 ? left0 : left1, w4.x, w4.y, w4.z};
                const float uv[4] = {up.x, up.y, up.z, up.w};
                const float zv[4] = {zp.x, zp.y, zp.z, zp.w};
                const bool ylo = h == 0 ? ylo0 : ylo1;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float w = wv[u];
                    float dx = w - lf[u], dy = w - uv[u], dz = w - zv[u];
                    if (FACES) {  // a low face's edge to the ghost is its own face term below
                        if (u == 0 && xlo0) dx = 0.f;
                        if (ylo) dy = 0.f;
                        if (p == 0) dz = 0.f;
                    }
                    tx = fmaf(dx, dx, tx);
                    ty = fmaf(dy, dy, ty);
                    tz = fmaf(dz, dz, tz);
                    tn = fmaf(w, w, tn);
                }
                float* dst = a.W + woff + (h == 0 ? 0 : nx);
                *reinterpret_cast<float4*>(dst) = w4;
                if (!FACES) {
                    // edges from the high faces to the zero ghost points
                    const float gy = ((h == 0 ? yhi0 : yhi1) ? ky : 0.f) + (zhi ? kz : 0.f);
                    if (gy != 0.f || xhi3) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float gc = gy + ((u == 3 && xhi3) ? kx : 0.f);
                            tg = fmaf(gc * wv[u], wv[u], tg);
                        }
                    }
                } else {
                    // every face: gamma_f w^2
                    const float gy = ((h == 0 ? yhi0 : yhi1) ? a.gam[3] : 0.f) + (ylo ? a.gam[2] : 0.f) +
                                     (zhi ? a.gam[5] : 0.f) + (p == 0 ? a.gam[4] : 0.f);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float gc = gy + ((u == 3 && xhi3) ? a.gam[1] : 0.f) + ((u == 0 && xlo0) ? a.gam[0] : 0.f);
                        if (gc != 0.f) tg = fmaf(gc * wv[u], wv[u], tg);
                    }
                }
            }
            two_sum_acc(an_hi, an_lo, tn);
            two_sum_acc(ae_hi, ae_lo, kx * tx + ky * ty + kz * tz + tg);
        }
        zp0 = w2[0];
        zp1 = w2[1];
        woff += plane;
        sbm = sbc;
        sbc = sbp;
        sbp = sbp + 1 == RB ? 0 : sbp + 1;
        sac = sac + 1 == RA ? 0 : sac + 1;
        if (++sst == DEPTH) {
            sst = 0;
            sph ^= 1u;
        }
    }
    if (abort_flag) {
        // drain this CTA's outstanding copies (bounded), report the timeout
        if (t == 0) {
            atomicOr(&a.st->status, 1);
            if (pfail == p0) mbar_wait(bars + DEPTH, 0);
            for (int q = pfail; q <= issued_upto; ++q)
                mbar_wait(bars + ((q - p0) % DEPTH), (unsigned)(((q - p0) / DEPTH) & 1));
        }
        __syncthreads();
        return false;
    }
    sum_n = (double)an_hi + (double)an_lo;
    sum_e = (double)ae_hi + (double)ae_lo;
    return true;
}


template <bool FIRST, int LGN, bool FACES>
__global__ void __launch_bounds__(FNT, 2) k_lanczos_fused_tma(const __grid_constant__ CUtensorMap mapB,
                                                             const __grid_constant__ CUtensorMap mapS,
                                                             const __grid_constant__ CUtensorMap mapA,
                                                             const __grid_constant__ CUtensorMap mapBn,
                                                             const __grid_constant__ CUtensorMap mapAn,
                                                             FusedArgs a) {
    if (a.st->done) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ double shred[FNT / 32];
    __shared__ int flag, abort_flag;
    const int t = threadIdx.x;
    // 1-D grid, z chunk major: per chunk the full-width tiles (x fastest,
    // then y) and then the narrow tiles of the last x columns, so the columns
    // both read are still in L2
    const int bid = blockIdx.x;
    const int per_z = a.nbx * a.nby + a.nby_s;
    const int tz = bid / per_z, q = bid - tz * per_z;
    double sum_n, sum_e;
    bool ok;
    if (q < a.nbx * a.nby)
        ok = fused_tile<FIRST, 5, FACES>(&mapB, &mapS, &mapA, a, q % a.nbx, q / a.nbx, tz, sm, abort_flag, sum_n,
                                         sum_e);
    else
        ok = fused_tile<FIRST, LGN, FACES>(&mapBn, &mapS, &mapAn, a, a.nbx, q - a.nbx * a.nby, tz, sm, abort_flag,
                                           sum_n, sum_e);
    if (!ok) return;
    const double alpha = a.H[(int64_t)a.j * a.m + a.j];

    // ---- deterministic grid reduction of (w.w, -w.Aw)
    const double d_nrm = block_sum<FNT>(sum_n, shred);
    const double d_edg = block_sum<FNT>(sum_e, shred);
    const int64_t nb = gridDim.x;
    const int64_t slot = bid;
    if (t == 0) a.red.partials[nb + slot] = d_edg;
    if (!grid_arrive(d_nrm, a.red.partials, a.red.counter, slot, nb, &flag)) return;
    const double nw2 = grid_finish<FNT>(a.red.partials, nb, a.red.counter, shred);
    const double edg = grid_finish<FNT>(a.red.partials + nb, nb, a.red.counter, shred);
    __shared__ double snext;
    __shared__ int cont;
    if (t == 0) {
        const int j = a.j, m = a.m;
        const double beta = sqrt(nw2);
        a.H[(int64_t)(j + 1) * m + j] = beta;
        const double bj = FIRST ? 0.0 : a.H[(int64_t)j * m + (j - 1)];
        const double nav = sqrt(alpha * alpha + bj * bj + beta * beta);  // ||A v_j||
        if (!(beta > 1e-12 * nav) || !isfinite(beta) || !isfinite(edg)) {
            if (!isfinite(beta) || !isfinite(edg)) a.st->status |= KV_ST_NONFINITE;
            a.st->done = 1;
            a.st->m_used = j + 1;
            cont = 0;
        } else {
            a.st->s[j + 1] = 1.0 / beta;
            snext = 1.0 / beta;
            if (j + 1 < m) {
                a.H[(int64_t)j * m + (j + 1)] = beta;
                a.H[(int64_t)(j + 1) * m + (j + 1)] = -edg / nw2;  // alpha_{j+1}
            }
            cont = (j + 1 < m) ? 1 : 0;
        }
    }
    __syncthreads();
    if (!cont || a.cd.o > PROJ_INLINE_MAX) return;  // launch_project takes many rows
    for (int r = 0; r < a.cd.o; ++r) {
        double v = 0.0;
        for (int64_t e = a.cd.rp[r] + t; e < a.cd.rp[r + 1]; e += FNT)
            v += c_entry(a.cd, e, a.W, &a.st->status);
        v = block_sum<FNT>(v, shred);
        if (t == 0) a.P[(int64_t)r * a.m + (a.j + 1)] = snext * v;
    }
}

// ---------------------------------------------------------------- host side
PfnEncodeTiled tensor_map_encoder() {
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

int make_grid_map(CUtensorMap* m, void* base, int64_t nx, int64_t ny, int64_t nz, int elem_bytes, int box_w,
                  int box_h) {
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)nx * elem_bytes, (cuuint64_t)nx * ny * elem_bytes};
    cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = tensor_map_encoder()(m, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                      3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return KV_ECUDA;
    }
    return KV_OK;
}

// Whether the single-pass TMA iteration applies: FP32 grid, rows a multiple
// of 16 bytes (TMA stride rule), extents that fit int coordinates.
bool fused_tma_supported(const Prob* p) {
    const Sys* s = p->sys;
    if (s->kind != 0 || p->prec != KV_FP32) return false;
    const int64_t nx = s->dims[0], ny = s->ndim >= 2 ? s->dims[1] : 1, nz = s->ndim >= 3 ? s->dims[2] : 1;
    if (nx % 4 != 0 || nx >= ((int64_t)1 << 30) || ny >= ((int64_t)1 << 30) || nz >= ((int64_t)1 << 30))
        return false;
    return tensor_map_encoder() != nullptr;
}

static int make_map(CUtensorMap* m, void* base, const Sys* s, int box_w, int box_h) {
    const int64_t nx = s->dims[0], ny = s->ndim >= 2 ? s->dims[1] : 1, nz = s->ndim >= 3 ? s->dims[2] : 1;
    return make_grid_map(m, base, nx, ny, nz, 4, box_w, box_h);
}

// One-time shared-memory limit of the kernel (not allowed during capture).
int fused_prepare() {
    static bool attr_set = false;
    if (!attr_set) {
        const void* fns[] = {(const void*)k_lanczos_fused_tma<true, 2, false>,
                             (const void*)k_lanczos_fused_tma<true, 3, false>,
                             (const void*)k_lanczos_fused_tma<true, 4, false>,
                             (const void*)k_lanczos_fused_tma<false, 2, false>,
                             (const void*)k_lanczos_fused_tma<false, 3, false>,
                             (const void*)k_lanczos_fused_tma<false, 4, false>,
                             (const void*)k_lanczos_fused_tma<true, 2, true>,
                             (const void*)k_lanczos_fused_tma<true, 3, true>,
                             (const void*)k_lanczos_fused_tma<true, 4, true>,
                             (const void*)k_lanczos_fused_tma<false, 2, true>,
                             (const void*)k_lanczos_fused_tma<false, 3, true>,
                             (const void*)k_lanczos_fused_tma<false, 4, true>};
        for (const void* fn : fns)
            KV_CHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TOTAL));
        attr_set = true;
    }
    return KV_OK;
}

// Grid of one launch.  Full-width tiles cover 124 columns each; when 1 to 60
// columns remain after them, narrow tiles of 4G - 4 >= remainder columns
// (G = 4, 8 or 16) cover those instead of one more full-width tile that
// would compute mostly outside the grid.
struct FusedGrid {
    int nbx, nby, sg_log2, nby_s, zc, nzch;
    int64_t n_norm, n_narrow;
};

static FusedGrid fused_grid(const Sys* s) {
    const int64_t nx = s->dims[0], ny = s->ndim >= 2 ? s->dims[1] : 1, nz = s->ndim >= 3 ? s->dims[2] : 1;
    FusedGrid f{};
    const int64_t full = nx / TXI, rem = nx - full * TXI;
    f.sg_log2 = 0;
    if (rem == 0) {
        f.nbx = (int)full;
    } else if (rem <= 60) {
        f.nbx = (int)full;
        f.sg_log2 = rem <= 12 ? 2 : (rem <= 28 ? 3 : 4);
    } else {
        f.nbx = (int)full + 1;
    }
    f.nby = (int)((ny + TYI - 1) / TYI);
    const int64_t ty_n = f.sg_log2 ? 16 * (32 >> f.sg_log2) - 1 : 1;
    f.nby_s = f.sg_log2 ? (int)((ny + ty_n - 1) / ty_n) : 0;
    // z chunk: about 12 waves of 2 resident CTAs per SM, at least 16 planes;
    // a small grid that would not fill one wave that way gets shorter chunks
    // (at least 2 planes), enough of them for one wave
    const int64_t per_z = (int64_t)f.nbx * f.nby + f.nby_s;
    const int64_t slots = 152LL * 2;
    const int64_t target = slots * 12;
    int64_t nzc = (target + per_z - 1) / per_z;
    if (nzc < 1) nzc = 1;
    int64_t zc = (nz + nzc - 1) / nzc;
    if (zc < 16) zc = 16;
    if (zc > nz) zc = nz;
    if (per_z * ((nz + zc - 1) / zc) < slots) {
        const int64_t want = (slots + per_z - 1) / per_z;
        zc = std::max<int64_t>(2, (nz + want - 1) / want);
        if (zc > nz) zc = nz;
    }
    f.zc = (int)zc;
    f.nzch = (int)((nz + zc - 1) / zc);
    f.n_norm = (int64_t)f.nbx * f.nby * f.nzch;
    f.n_narrow = (int64_t)f.nby_s * f.nzch;
    return f;
}

int fused_tma_blocks(const Prob* p, int* zc_out) {
    const FusedGrid f = fused_grid(p->sys);
    *zc_out = f.zc;
    return (int)(f.n_norm + f.n_narrow);
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
    const FusedGrid f = fused_grid(s);
    // narrow tiles: 4G columns, 16 * 32/G rows of w (G = 4: 16 x 128)
    const int lg = f.sg_log2 ? f.sg_log2 : 2;
    const int wc_n = 4 << lg, wr_n = 16 * (32 >> lg);
    CUtensorMap mB, mS, mA, mBn, mAn;
    int rc = make_map(&mB, const_cast<void*>(B), s, BBW, BBH);
    if (!rc) rc = make_map(&mS, const_cast<void*>(B), s, SBW, SBH);
    if (!rc) rc = make_map(&mA, const_cast<void*>(A), s, ABW, ABH);
    if (!rc) rc = make_map(&mBn, const_cast<void*>(B), s, wc_n, wr_n + 2);
    if (!rc) rc = make_map(&mAn, const_cast<void*>(A), s, wc_n, wr_n);
    if (rc) return rc;
    const int64_t nblk = f.n_norm + f.n_narrow;
    if (nblk < 1 || nblk > INT32_MAX) {
        set_error("fused grid of %lld blocks", (long long)nblk);
        return KV_EINVAL;
    }
    dim3 grd((unsigned)nblk);
    FusedArgs a;
    a.W = (float*)Wout;
    a.g = g;
    a.zc = f.zc;
    a.nbx = f.nbx;
    a.nby = f.nby;
    a.sg_log2 = f.sg_log2;
    a.nby_s = f.nby_s;
    a.st = p->d_state + j;
    a.H = p->d_H + (int64_t)j * (p->m + 1) * p->m;
    a.P = p->d_P + (int64_t)j * p->o * p->m;
    a.cd = CDesc{p->o, p->d_crp, p->d_ccol, p->d_cval, p->N};
    a.m = p->m;
    a.j = it;
    a.red = p->red;
    {
        const double kap[3] = {g.kx, g.ky, g.kz};
        for (int f = 0; f < 6; ++f) {
            a.gam[f] = (float)s->face[f];
            a.rho[f] = (float)(kap[f >> 1] > 0.0 ? s->face[f] / kap[f >> 1] : 0.0);
        }
    }
    rc = fused_prepare();
    if (rc) return rc;
    LaunchScope ls(p->ctx, "lanczos_fused");
    cudaStream_t st = p->ctx->stream;
    // the narrow shape is a template argument (G = 4 when there are none:
    // that branch is then never taken)
    auto go = [&](auto first, auto lgn) {
        if (s->faces)
            k_lanczos_fused_tma<decltype(first)::value, decltype(lgn)::value, true>
                <<<grd, FNT, SMEM_TOTAL, st>>>(mB, mS, mA, mBn, mAn, a);
        else
            k_lanczos_fused_tma<decltype(first)::value, decltype(lgn)::value, false>
                <<<grd, FNT, SMEM_TOTAL, st>>>(mB, mS, mA, mBn, mAn, a);
    };
    using T = std::true_type;
    using F = std::false_type;
    using L2 = std::integral_constant<int, 2>;
    using L3 = std::integral_constant<int, 3>;
    using L4 = std::integral_constant<int, 4>;
    if (it == 0) {
        if (lg == 2) go(T{}, L2{});
        else if (lg == 3) go(T{}, L3{});
        else go(T{}, L4{});
    } else {
        if (lg == 2) go(F{}, L2{});
        else if (lg == 3) go(F{}, L3{});
        else go(F{}, L4{});
    }
    KV_CHECK_CUDA(cudaGetLastError());
    return KV_OK;
}

// One block waits on an mbarrier nothing arrives on, with the kernel's own
// bounded-wait routine: the wait must expire and is recorded in *status.
__global__ void k_diag_wait(unsigned* status, long polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, polls);
    if (!ok) atomicOr(status, 1u);
}

}  // namespace kv

extern "C" int kv_diag_bounded_wait(int device, int64_t polls) {
    using namespace kv;
    if (polls < 1 || polls > WAIT_LIMIT) {
        set_error("kv_diag_bounded_wait: polls must be in [1, %ld]", WAIT_LIMIT);
        return KV_EINVAL;
    }
    DeviceGuard dg(device);
    if (dg.err != cudaSuccess) {
        set_error("kv_diag_bounded_wait: device %d", device);
        return KV_EINVAL;
    }
    unsigned* d_status = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        k_diag_wait<<<1, 32, 0, st>>>(d_status, (long)polls);
        e = cudaGetLastError();
    }
    unsigned h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d_status) cudaFree(d_status);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        set_error("kv_diag_bounded_wait: %s", cudaGetErrorString(e));
        return KV_ECUDA;
    }
    if (h) {
        set_error("kv_diag_bounded_wait: the wait expired after %lld polls", (long long)polls);
        return KV_ETIMEOUT;
    }
    return KV_OK;
}
