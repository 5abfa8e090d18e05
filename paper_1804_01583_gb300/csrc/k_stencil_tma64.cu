// k_stencil_tma64.cu -- single-pass Lanczos iteration on the grid operator in
// FP64 (FP64 storage of the Krylov vectors, FP64 arithmetic for the vectors).
//
// One launch performs iteration j of the projected Lanczos loop (Alg. 3 with
// the Alg. 4 projection), like the FP32 kernel of k_stencil_tma.cu:
//     w = A v_j - alpha_j v_j - beta_j v_{j-1}           (written to a third buffer)
//     beta_{j+1}^2 = w . w,  alpha_{j+1} = (w . A w) / (w . w)
//     P[:, j+1] = C w / beta_{j+1}
// so each iteration reads v_j and v_{j-1} once and writes w once: 24 bytes a
// grid point, the minimum of a three-vector FP64 Lanczos step.
//
// Where the time goes on this GPU: its FP64 pipe retires about two FP64
// instructions per SM per clock (1/64 of FP32), so an FP64 iteration is bound
// by its FP64 instruction count, not by HBM.  The vector w itself is computed
// with FP64 instructions: 8 a point for the 7-point update (three
// neighbour-pair sums, one multiply, four fused multiply-adds), or 7 in the
// unit form, which stores w divided by s_j kappa_x (s_j the lazy scale of
// v_j's buffer) so that the x pair needs no multiply; the factor enters
// beta_{j+1} and the buffer's scale.  The two sums that need no FP64 result
// per point are taken off the FP64 pipe:
//   - each w is split exactly into three floats (a1 + a2 + a3 = w, by integer
//     operations on its bits: 24 + 23 + 6 significant bits);
//   - w . w and the summation-by-parts form of w . A w,
//         w . A w = - sum_a kappa_a sum_edges (w_p - w_q)^2 - sum_faces gamma_f sum w_p^2,
//     are accumulated with error-free float transformations (TwoSum,
//     TwoProduct by FMA), the differences w_p - w_q formed from the exact
//     splits, so every term keeps about 47 significant bits and the sums are
//     compensated; per-thread sums become doubles once at the end.
//
// Grid boundary: each face f of the box grid has a coefficient gamma_f >= 0,
// and a point on face f gets -gamma_f v_p in place of the coupling to the
// missing neighbour: gamma = kappa_a (= coef / h_a^2) is the Dirichlet-0
// boundary of the vertex grid, gamma = 0 an insulated face, anything between
// a heat exchange (Sec. 5.3).  TMA reads zeros outside the grid (the
// Dirichlet ghost); other faces add s_j (kappa_a - gamma_f) v_p at their
// points.
//
// Tiling: a CTA owns 126 (x) x 15 (y) points and marches over a chunk of z
// planes.  w is evaluated on a 128 x 16 region (x0-2 .. x0+125, y0-1 ..
// y0+14: the tile plus the low-x and low-y neighbours its backward differences
// need); warp k owns rows 2k and 2k+1, lane l the columns 2l, 2l+1, 64+2l
// and 65+2l, so every 16-byte load or store of a warp covers 512 contiguous
// bytes (shared memory without bank conflicts, whole global sectors).  v_j
// arrives by TMA (a 128 x 18 box and a 2-column side box for the x0+126
// neighbour) in a ring two planes ahead, v_{j-1} by plain coalesced loads one
// plane ahead.  Each plane of w also goes to a double-buffered shared plane,
// and the sums of a plane run one iteration later from that copy (the z-1
// split stays in registers), interleaved with the next plane's FP64 work:
// every warp's instruction stream then mixes FP64 and float work, and the
// FP64 pipe does not idle while the float sums run.
//
// Every mbarrier wait is bounded; on expiry the CTA sets the column's status
// word (reported as KV_ETIMEOUT), drains its outstanding copies with bounded
// waits and leaves.
#include <cuda.h>
#include <stdlib.h>

#include <type_traits>

#include "kv_internal.h"
#include "reduce.cuh"
#include "splits.cuh"
#include "tma.cuh"

namespace kv {

constexpr int DNT = 256;
constexpr int DTX = 126, DTY = 15;      // interior points of a tile
constexpr int DWC = 128, DWR = 16;      // w region: x0-2 .. x0+125, y0-1 .. y0+14
constexpr int DBW = 128, DBH = 18;      // v_j box: x0-2 .. x0+125, y0-2 .. y0+15 (1 KB rows)
constexpr int DSW = 2;                  // v_j side box: x0+126 .. x0+127, same rows
constexpr int DDEPTH = 2;               // planes of v_j in flight ahead of the compute
constexpr int DRB = DDEPTH + 2;         // ring slots: planes p-1 .. p+DDEPTH
constexpr int DBBYTES = DBW * DBH * 8;  // 18432
constexpr int DSBYTES = DSW * DBH * 8;  // 288
constexpr int DSSTRIDE = 384;
constexpr int DWPLANE = DWC * DWR * 8;  // one plane of w (doubles), kept for the next iteration's sums
constexpr int DSMEM_MAIN = DRB * (DBBYTES + DSSTRIDE) + 2 * DWPLANE;
constexpr int DSMEM_TOTAL = DSMEM_MAIN + 128 + 1024;  // + barriers + alignment slack

// ------------------------------------------------------------------ kernel --
struct Fused64Args {
    double* W;          // output buffer: w (unnormalised v_{j+1}), or w / (s_j kappa_x) in the unit form
    const double* Aprev;  // v_{j-1} (unnormalised; unused in the first iteration)
    StencilGeom g;
    double gface[6];    // gamma per face: x low, x high, y low, y high, z low, z high
    float gfh[6], gfl[6];  // the same as float pairs (gamma = gfh + gfl to 2^-48), the face terms' weights
    double kmg[6];      // kappa_axis - gamma per face: a face point adds s_j (kappa - gamma) v_p to w
    double kmgx[6];     // the same divided by kappa_x, for the unit form
    double ry, rz;      // kappa_y / kappa_x, kappa_z / kappa_x (unit form)
    double ikx;         // 1 / kappa_x (unit form)
    double wbound;      // bound of |w| for a unit v_j (4 sum |kappa| + sum gamma >= ||A||_2)
    int unit_ok;        // the unit form may be used (kappa_x > 0, bounded drift)
    int zc;             // z planes per CTA
    int nbx, nby;       // tiles per z chunk: nbx x nby
    ColState* st;
    double* H;          // this column's (m+1) x m
    double* P;          // this column's o x m
    CDesc cd;
    int m, j;
    Reduce red;
};

// Whether iteration j stores w' = w / (s_j kappa_x) (7 FP64 instructions a
// point) or w itself (8).  In the unit form each stored buffer is the previous
// one times beta_{j+1} / kappa_x, so the buffers' magnitudes drift by up to
// log2(3 wbound / kappa_x) bits an iteration (the host allows the form only
// below 64); once s_j kappa_x leaves (2^-250, 2^250) one iteration stores w,
// whose norm is beta_{j+1}, and the drift starts again from there.  Every
// thread of the launch reads the same s_j, so the choice is uniform.
__device__ __forceinline__ bool fused64_unit(const Fused64Args& a) {
    const double f = a.st->s[a.j] * a.g.kx;
    return a.unit_ok && f > 0x1p-250 && f < 0x1p250;
}

// The point's face flags: bit 2a for the low face of axis a, 2a+1 for the high.
__device__ __forceinline__ unsigned face_bits(int x, int y, int z, int nx, int ny, int nz) {
    return (x == 0 ? 1u : 0u) | (x == nx - 1 ? 2u : 0u) | (y == 0 ? 4u : 0u) | (y == ny - 1 ? 8u : 0u) |
           (z == 0 ? 16u : 0u) | (z == nz - 1 ? 32u : 0u);
}

// One CTA's tile and chunk of z planes.  Returns false when a stage wait
// expired (the copies are drained and the timeout reported); otherwise this
// thread's sums: sum_n = w . w and sum_e = -(w . A w), as doubles.
template <bool FIRST, bool FACES, bool UNIT>
__device__ __forceinline__ bool fused64_tile(const CUtensorMap* mB, const CUtensorMap* mS, const Fused64Args& a,
                                             int tx, int ty, int tz, unsigned char* sm, int& abort_flag,
                                             double& sum_n, double& sum_e) {
    double* sB = (double*)sm;
    double* sS = (double*)(sm + DRB * DBBYTES);
    double* sW = (double*)(sm + DRB * (DBBYTES + DSSTRIDE));
    uint64_t* bars = (uint64_t*)(sm + DSMEM_MAIN);  // DDEPTH stage barriers + 1 prologue barrier
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const StencilGeom& g = a.g;
    const int nx = (int)g.nx, ny = (int)g.ny, nz = (int)g.nz;
    const int x0 = tx * DTX, y0 = ty * DTY;
    const int z0 = tz * a.zc;
    const int z1 = min(z0 + a.zc, nz);
    const int p0 = z0 - 1;  // w planes p0 .. z1-1; the sums run over z0 .. z1-1
    constexpr unsigned stage_bytes = (unsigned)(DBBYTES + DSBYTES);

    // w = s_j A v_j - alpha_j s_j v_j - beta_j s_{j-1} v_{j-1} in the
    // pair-sum form fx (l + r) + fy (d + u) + fz (m + p) + fc c + fa a
    // (3 additions, a multiply and 4 FMAs), or in the unit form divided by
    // fx = s_j kappa_x: (l + r) + ry (d + u) + rz (m + p) + rc c + ra a
    // (3 additions and 4 FMAs); the factor then goes into beta_{j+1} and the
    // scale of the stored buffer (Alg. 3's normalisation, applied lazily)
    const double sj = a.st->s[a.j];
    const double alpha = a.H[(int64_t)a.j * a.m + a.j];
    const double fx = sj * g.kx;
    const double fa = FIRST ? 0.0 : -a.H[(int64_t)a.j * a.m + (a.j - 1)] * a.st->s[a.j - 1];
    const double cy = UNIT ? a.ry : sj * g.ky;
    const double cz = UNIT ? a.rz : sj * g.kz;
    const double cc0 = UNIT ? (g.kc - alpha) * a.ikx : sj * (g.kc - alpha);
    const double ca = UNIT ? fa / fx : fa;
    // split scale: |stored w| 2^-sh < 2^8, from |w| <= wbound (3 wbound with
    // the orthogonality the recurrence has lost)
    int sh = 1;
    {
        const double q = UNIT ? a.wbound / fx : a.wbound;
        int e = 0;
        if (q > 0.0 && q < INFINITY) frexp(q, &e);  // q < 2^e
        sh = e + 1;
    }

    auto ring = [](int plane) { return ((plane % DRB) + DRB) % DRB; };
    auto load_b = [&](int plane, uint64_t* bar) {  // v_j plane: main box + side box, same ring slot
        const int k = ring(plane);
        tma_load_3d(sB + (size_t)k * (DBBYTES / 8), mB, bar, x0 - 2, y0 - 2, plane);
        tma_load_3d(sS + (size_t)k * (DSSTRIDE / 8), mS, bar, x0 + DTX, y0 - 2, plane);
    };

    // this thread's points: region rows r0, r0 + 1 (y = y0 - 1 + r), region
    // columns 2 lane, 2 lane + 1, 64 + 2 lane, 65 + 2 lane (x = x0 - 2 + column)
    const int r0 = 2 * warp;
    const int yr[2] = {y0 - 1 + r0, y0 + r0};
    int xu[4];
    bool xin[4], xint[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = (u < 2 ? 0 : 64) + 2 * lane + (u & 1);
        xu[u] = x0 - 2 + c;
        xin[u] = xu[u] >= 0 && xu[u] < nx;
        xint[u] = xin[u] && c >= 2;  // interior columns: x >= x0
    }
    const bool yin[2] = {yr[0] >= 0 && yr[0] < ny, yr[1] < ny};
    const bool yint[2] = {yin[0] && r0 >= 1, yin[1]};

    if (t == 0) {
        for (int q = 0; q <= DDEPTH; ++q) mbar_init(bars + q, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    int issued_upto = p0 - 1;
    if (t == 0) {
        uint64_t* pro = bars + DDEPTH;
        mbar_expect_tx(pro, 2 * stage_bytes);
        load_b(p0 - 1, pro);
        load_b(p0, pro);
        for (int q = 0; q < DDEPTH && p0 + q <= z1 - 1; ++q) {  // stage q: B(q+1)
            uint64_t* bar = bars + q;
            mbar_expect_tx(bar, stage_bytes);
            load_b(p0 + q + 1, bar);
            issued_upto = p0 + q;
        }
    }

    // v_{j-1} at this thread's points of plane p (plain loads, one plane ahead)
    const int64_t plane = (int64_t)nx * ny;
    double2 an[2][2];
    auto load_a = [&](int p) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < 2; ++k) an[h][k] = make_double2(0.0, 0.0);
        if constexpr (!FIRST) {  // the first iteration has no v_{j-1}
            if (p < 0 || p >= nz) return;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!yin[h]) continue;
                const double* row = a.Aprev + (int64_t)p * plane + (int64_t)yr[h] * nx;
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (xin[2 * k]) an[h][k] = __ldcs(reinterpret_cast<const double2*>(row + xu[2 * k]));
            }
        }
    };
    load_a(p0);

    F3 prev[2][4];  // split of w at plane q-1 while the sums of plane q run
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int u = 0; u < 4; ++u) prev[h][u] = F3{0.f, 0.f, 0.f};
    Acc2 acc_n, acc_x, acc_y, acc_z;
    Acc2 acc_g;  // FACES: sum of gamma_f w^2 over the faces' points
    int pfail = -1;
    int sbm = ring(p0 - 1), sbc = ring(p0), sbp = ring(p0 + 1), sst = 0;
    unsigned sph = 0;
    // Iteration p computes w on plane p (FP64) and, from the copy of w kept in
    // shared memory, the sums of plane q = p - 1 (float and integer work), so
    // each warp's instruction stream mixes both and the FP64 pipe stays fed.
    // One more iteration after the last plane finishes its sums.
    for (int p = p0; p <= z1; ++p) {
        const bool wplane = p <= z1 - 1;
        bool ok = true;
        if (wplane) {
            if (p == p0) ok = mbar_wait(bars + DDEPTH, 0);
            ok = ok && mbar_wait(bars + sst, sph);
        }
        // No barrier here: each thread's own wait makes the stage visible to
        // it; a failed wait is acted on after the barrier below.
        if (!ok) abort_flag = 1;
        const double* Bm = sB + (size_t)sbm * (DBBYTES / 8);
        const double* Bc = sB + (size_t)sbc * (DBBYTES / 8);
        const double* Bp = sB + (size_t)sbp * (DBBYTES / 8);
        const double* Sc = sS + (size_t)sbc * (DSSTRIDE / 8);
        double* Wp = sW + (p & 1) * (DWC * DWR);           // w of plane p (written here)
        const double* Wq = sW + ((p + 1) & 1) * (DWC * DWR);  // w of plane q = p - 1
        const bool pin = p >= 0 && p < nz;
        const int qz = p - 1;

#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = r0 + h;  // region row; box row r + 1 is its own y
            // ---- w of plane p on row r (FP64)
            if (wplane) {
                double cc[4], dd[4], uu[4], mm[4], pp[4];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int c0 = 64 * k + 2 * lane;
                    const double2 c2 = *reinterpret_cast<const double2*>(Bc + (r + 1) * DBW + c0);
                    const double2 d2 = *reinterpret_cast<const double2*>(Bc + r * DBW + c0);
                    const double2 u2 = *reinterpret_cast<const double2*>(Bc + (r + 2) * DBW + c0);
                    const double2 m2 = *reinterpret_cast<const double2*>(Bm + (r + 1) * DBW + c0);
                    const double2 p2 = *reinterpret_cast<const double2*>(Bp + (r + 1) * DBW + c0);
                    cc[2 * k] = c2.x, cc[2 * k + 1] = c2.y;
                    dd[2 * k] = d2.x, dd[2 * k + 1] = d2.y;
                    uu[2 * k] = u2.x, uu[2 * k + 1] = u2.y;
                    mm[2 * k] = m2.x, mm[2 * k + 1] = m2.y;
                    pp[2 * k] = p2.x, pp[2 * k + 1] = p2.y;
                }
                // x neighbours: column 2l+2 is lane l+1's first point (lane 0's
                // third for lane 31), column 63+2l lane l-1's fourth (lane 31's
                // second for lane 0), column 66+2l lane l+1's third (the side box
                // for lane 31); lane 0's first left value only feeds w(x0-2),
                // which nothing uses
                const double l0 = __shfl_up_sync(0xffffffffu, cc[1], 1);
                const double r1 = __shfl_sync(0xffffffffu, lane == 0 ? cc[2] : cc[0], (lane + 1) & 31);
                const double l2 = __shfl_sync(0xffffffffu, lane == 31 ? cc[1] : cc[3], (lane + 31) & 31);
                double r3 = __shfl_down_sync(0xffffffffu, cc[2], 1);
                if (lane == 31) r3 = Sc[(r + 1) * DSW];
                const double xl[4] = {l0, cc[0], l2, cc[2]};
                const double xr[4] = {cc[1], r1, cc[3], r3};
                const double aa[4] = {an[h][0].x, an[h][0].y, an[h][1].x, an[h][1].y};
                double wv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    double w = xl[u] + xr[u];
                    if (!UNIT) w *= fx;
                    w = fma(cy, dd[u] + uu[u], w);
                    w = fma(cz, mm[u] + pp[u], w);
                    w = fma(cc0, cc[u], w);
                    if (!FIRST) w = fma(ca, aa[u], w);
                    if (FACES) {
                        const unsigned fb = face_bits(xu[u], yr[h], p, nx, ny, nz);
                        if (fb) {  // a point on face f adds s_j (kappa - gamma_f) c (over fx: unit form)
                            double d = 0.0;
#pragma unroll
                            for (int f = 0; f < 6; ++f)
                                if (fb & (1u << f)) d += UNIT ? a.kmgx[f] : a.kmg[f];
                            w = fma(UNIT ? d : sj * d, cc[u], w);
                        }
                    }
                    wv[u] = (pin && yin[h] && xin[u]) ? w : 0.0;
                }
                // interior points of planes z0.. go to memory (pairs are inside
                // or outside the grid together: nx is even)
                if (p >= z0 && yint[h]) {
                    double* row = a.W + (int64_t)p * plane + (int64_t)yr[h] * nx;
                    if (xint[0]) *reinterpret_cast<double2*>(row + xu[0]) = make_double2(wv[0], wv[1]);
                    if (xint[2]) *reinterpret_cast<double2*>(row + xu[2]) = make_double2(wv[2], wv[3]);
                }
                *reinterpret_cast<double2*>(Wp + r * DWC + 2 * lane) = make_double2(wv[0], wv[1]);
                *reinterpret_cast<double2*>(Wp + r * DWC + 64 + 2 * lane) = make_double2(wv[2], wv[3]);
            }
            // ---- the sums of plane q = p - 1 on row r (float and integer work)
            if (qz >= p0) {
                F3 cur[4];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const double2 v2 = *reinterpret_cast<const double2*>(Wq + r * DWC + 64 * k + 2 * lane);
                    cur[2 * k] = split3(v2.x, sh);
                    cur[2 * k + 1] = split3(v2.y, sh);
                }
                if (qz >= z0 && yint[h]) {
                    // x-1: column 2l-1 is lane l-1's second point, column 63+2l
                    // lane l-1's fourth (lane 31's second for lane 0); y-1: the row
                    // below (another warp's row for h = 0); z-1: plane q-1
                    F3 left[4], up[4];
                    left[1] = cur[0];
                    left[3] = cur[2];
                    left[0].a1 = __shfl_up_sync(0xffffffffu, cur[1].a1, 1);
                    left[0].a2 = __shfl_up_sync(0xffffffffu, cur[1].a2, 1);
                    left[0].a3 = __shfl_up_sync(0xffffffffu, cur[1].a3, 1);
                    const F3 snd = lane == 31 ? cur[1] : cur[3];
                    left[2].a1 = __shfl_sync(0xffffffffu, snd.a1, (lane + 31) & 31);
                    left[2].a2 = __shfl_sync(0xffffffffu, snd.a2, (lane + 31) & 31);
                    left[2].a3 = __shfl_sync(0xffffffffu, snd.a3, (lane + 31) & 31);
                    if (h == 1) {
                        // row r0 of plane q: its split has just been kept in prev[0]
#pragma unroll
                        for (int u = 0; u < 4; ++u) up[u] = prev[0][u];
                    } else {
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const double2 v2 =
                                *reinterpret_cast<const double2*>(Wq + (r - 1) * DWC + 64 * k + 2 * lane);
                            up[2 * k] = split3(v2.x, sh);
                            up[2 * k + 1] = split3(v2.y, sh);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (!xint[u]) continue;
                        const F3 w = cur[u];
                        float nh, nl, th, tl;
                        sq3(w, nh, nl);
                        acc_n.add(nh, nl);
                        unsigned fb = 0;
                        if (FACES) fb = face_bits(xu[u], yr[h], qz, nx, ny, nz);
                        // backward edges; on a low face the edge to the zero ghost
                        // is the Dirichlet term, replaced by the face's own one
                        if (!FACES || !(fb & 1u)) {
                            sqdiff3(w, left[u], th, tl);
                            acc_x.add(th, tl);
                        }
                        if (!FACES || !(fb & 4u)) {
                            sqdiff3(w, up[u], th, tl);
                            acc_y.add(th, tl);
                        }
                        if (!FACES || !(fb & 16u)) {
                            sqdiff3(w, prev[h][u], th, tl);
                            acc_z.add(th, tl);
                        }
                        if (!FACES) {
                            // Dirichlet high faces: the edge to the zero ghost, weight kappa
                            if (xu[u] == nx - 1) acc_x.add(nh, nl);
                            if (yr[h] == ny - 1) acc_y.add(nh, nl);
                            if (qz == nz - 1) acc_z.add(nh, nl);
                        } else if (fb) {
                            // gamma_f w^2 with gamma as a float pair: the product
                            // keeps about 47 bits, like every other term
#pragma unroll
                            for (int f = 0; f < 6; ++f)
                                if (fb & (1u << f)) {
                                    const float gh = a.gfh[f], gl = a.gfl[f];
                                    const float pp = __fmul_rn(gh, nh);
                                    const float pe = __fmaf_rn(gh, nh, -pp);
                                    acc_g.add(pp, __fmaf_rn(gh, nl, __fmaf_rn(gl, nh, pe)));
                                }
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) prev[h][u] = cur[u];
            }
        }
        if (wplane) load_a(p + 1);  // v_{j-1} of the next plane, in flight meanwhile
        __syncthreads();  // w of plane p visible; plane q's copy and B(p-1) no longer read
        if (abort_flag) {  // some thread's wait expired: the stage may be incomplete
            pfail = p;
            break;
        }
        if (t == 0 && p + DDEPTH <= z1 - 1) {
            // stage p + DDEPTH reuses this stage's barrier and B(p-1)'s slot
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int q = p + DDEPTH;
            uint64_t* bar = bars + sst;
            mbar_expect_tx(bar, stage_bytes);
            load_b(q + 1, bar);
            issued_upto = q;
        }
        sbm = sbc;
        sbc = sbp;
        sbp = sbp + 1 == DRB ? 0 : sbp + 1;
        if (++sst == DDEPTH) {
            sst = 0;
            sph ^= 1u;
        }
    }
    if (abort_flag) {
        // drain this CTA's outstanding copies (bounded), report the timeout
        if (t == 0) {
            atomicOr(&a.st->status, 1);
            if (pfail == p0) mbar_wait(bars + DDEPTH, 0);
            for (int q = pfail; q <= issued_upto; ++q)
                mbar_wait(bars + ((q - p0) % DDEPTH), (unsigned)(((q - p0) / DDEPTH) & 1));
        }
        __syncthreads();
        return false;
    }
    const double s2 = ldexp(1.0, 2 * sh);
    sum_n = acc_n.value() * s2;
    double e = g.kx * acc_x.value() + g.ky * acc_y.value() + g.kz * acc_z.value();
    if (FACES) e += acc_g.value();
    sum_e = e * s2;
    return true;
}

template <bool FIRST, bool FACES>
__global__ void __launch_bounds__(DNT, 2) k_lanczos_fused64(const __grid_constant__ CUtensorMap mapB,
                                                           const __grid_constant__ CUtensorMap mapS,
                                                           Fused64Args a) {
    dep_wait();  // the previous iteration's w, scalars and state are complete
    if (a.st->done) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ double shred[DNT / 32];
    __shared__ int flag, abort_flag;
    const int t = threadIdx.x;
    // 1-D grid, z chunk major; per chunk nbx x nby tiles, x fastest
    const int bid = blockIdx.x;
    const int per_z = a.nbx * a.nby;
    const int tz = bid / per_z, q = bid - tz * per_z;
    double sum_n, sum_e;
    const bool unit = fused64_unit(a);
    const bool ran = unit ? fused64_tile<FIRST, FACES, true>(&mapB, &mapS, a, q % a.nbx, q / a.nbx, tz, sm, abort_flag,
                                                             sum_n, sum_e)
                          : fused64_tile<FIRST, FACES, false>(&mapB, &mapS, a, q % a.nbx, q / a.nbx, tz, sm,
                                                              abort_flag, sum_n, sum_e);
    if (!ran) return;
    const double alpha = a.H[(int64_t)a.j * a.m + a.j];

    // ---- deterministic grid reduction of (w.w, -w.Aw)
    const double d_nrm = block_sum<DNT>(sum_n, shred);
    const double d_edg = block_sum<DNT>(sum_e, shred);
    const int64_t nb = gridDim.x;
    const int64_t slot = bid;
    if (t == 0) a.red.partials[nb + slot] = d_edg;
    if (!grid_arrive(d_nrm, a.red.partials, a.red.counter, slot, nb, &flag)) return;
    // the last CTA: every other CTA has finished, so the next launch may be
    // scheduled (its CTAs wait in dep_wait until this grid has completed)
    dep_release();
    const double nw2 = grid_finish<DNT>(a.red.partials, nb, a.red.counter, shred);
    const double edg = grid_finish<DNT>(a.red.partials + nb, nb, a.red.counter, shred);
    __shared__ double snext;
    __shared__ int cont;
    if (t == 0) {
        const int j = a.j, m = a.m;
        // nw2 and edg: w.w and -w.A w for the stored vector (w, or w / fx)
        const double nrm = sqrt(nw2);
        const double beta = unit ? a.st->s[j] * a.g.kx * nrm : nrm;  // ||w||
        a.H[(int64_t)(j + 1) * m + j] = beta;
        const double bj = FIRST ? 0.0 : a.H[(int64_t)j * m + (j - 1)];
        const double nav = sqrt(alpha * alpha + bj * bj + beta * beta);  // ||A v_j||
        if (!(beta > 1e-12 * nav) || !isfinite(beta) || !isfinite(edg)) {
            if (!isfinite(beta) || !isfinite(edg)) a.st->status |= KV_ST_NONFINITE;
            a.st->done = 1;
            a.st->m_used = j + 1;
            cont = 0;
        } else {
            a.st->s[j + 1] = 1.0 / nrm;  // v_{j+1} = stored / ||stored||
            snext = 1.0 / nrm;
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
        for (int64_t e = a.cd.rp[r] + t; e < a.cd.rp[r + 1]; e += DNT)
            v += c_entry(a.cd, e, a.W, &a.st->status);
        v = block_sum<DNT>(v, shred);
        if (t == 0) a.P[(int64_t)r * a.m + (a.j + 1)] = snext * v;
    }
}

// ---------------------------------------------------------------- host side
// Whether the single-pass FP64 iteration applies: FP64 grid, rows a multiple
// of 16 bytes (TMA stride rule: nx even), extents that fit int coordinates,
// and at least FUSED64_MIN_POINTS points.  Its float-split sums keep about 47
// bits a term, so alpha and beta carry relative errors near 1e-14 at any
// size; plain FP64 dot products (the two-pass kernels) are more accurate
// below a few thousand points, and on such small grids an exhausted Krylov
// space (beta at rounding level, Alg. 3's breakdown) is told apart from a
// continuing one only at that accuracy.  The fused kernel gains nothing
// there: a grid that small is one partial wave of tiles.
constexpr int64_t FUSED64_MIN_POINTS = 4096;

bool fused64_supported(const Prob* p) {
    const Sys* s = p->sys;
    if (s->kind != 0 || p->prec != KV_FP64) return false;
    if (s->n < FUSED64_MIN_POINTS) return false;
    const int64_t nx = s->dims[0], ny = s->ndim >= 2 ? s->dims[1] : 1, nz = s->ndim >= 3 ? s->dims[2] : 1;
    if (nx % 2 != 0 || nx >= ((int64_t)1 << 30) || ny >= ((int64_t)1 << 30) || nz >= ((int64_t)1 << 30))
        return false;
    return tensor_map_encoder() != nullptr;
}

int fused64_prepare() {
    static bool attr_set = false;
    if (!attr_set) {
        const void* fns[] = {(const void*)k_lanczos_fused64<true, false>, (const void*)k_lanczos_fused64<false, false>,
                             (const void*)k_lanczos_fused64<true, true>, (const void*)k_lanczos_fused64<false, true>};
        for (const void* fn : fns)
            KV_CHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, DSMEM_TOTAL));
        attr_set = true;
    }
    return KV_OK;
}

// Grid of one launch: tiles of 126 x 15 points, z chunks of zc planes.  Each
// chunk also computes w on the plane below it (the z-1 differences) and pays
// a fixed start (barrier set-up, the first planes' copies, the reduction),
// about two planes' worth, so the chunk length trades those against the tail
// of the last wave: zc >= 2 minimises ceil(chunks x tiles / slots) x
// (zc + 3), with two resident CTAs per SM.
struct Fused64Grid {
    int nbx, nby, zc, nzch;
    int64_t blocks;
};

static Fused64Grid fused64_grid(const Sys* s, int sms) {
    const int64_t nx = s->dims[0], ny = s->ndim >= 2 ? s->dims[1] : 1, nz = s->ndim >= 3 ? s->dims[2] : 1;
    Fused64Grid f{};
    f.nbx = (int)((nx + DTX - 1) / DTX);
    f.nby = (int)((ny + DTY - 1) / DTY);
    const int64_t tiles = (int64_t)f.nbx * f.nby;
    const int64_t slots = 2LL * (sms > 0 ? sms : 152);
    int64_t best_zc = nz, best_cost = INT64_MAX;
    for (int64_t zc = std::min<int64_t>(2, nz); zc <= nz; ++zc) {
        const int64_t nch = (nz + zc - 1) / zc;
        if (zc > 2 && (nz + zc - 2) / (zc - 1) == nch) continue;  // same chunk count as zc - 1
        const int64_t waves = (nch * tiles + slots - 1) / slots;
        const int64_t cost = waves * (zc + 3);
        if (cost < best_cost) {
            best_cost = cost;
            best_zc = zc;
        }
    }
    // Within one wave the FP64 pipe of an SM is shared by its CTAs, so two
    // short chunks on one SM take as long as one chunk of twice the planes,
    // plus a second halo; count the CTAs per SM instead (a lone CTA keeps the
    // pipe less busy: taken as 0.8 of a pair's rate).
    if ((nz + best_zc - 1) / best_zc * tiles <= slots) {
        const int64_t sm = slots / 2;
        double best = 1e300;
        for (int64_t zc = std::min<int64_t>(2, nz); zc <= nz; ++zc) {
            const int64_t nch = (nz + zc - 1) / zc;
            if (zc > 2 && (nz + zc - 2) / (zc - 1) == nch) continue;
            const int64_t per = (nch * tiles + sm - 1) / sm;
            const double cost = (double)(per * (zc + 3)) / (per == 1 ? 0.8 : 1.0);
            if (cost < best) {
                best = cost;
                best_zc = zc;
            }
        }
    }
    f.zc = (int)best_zc;
    f.nzch = (int)((nz + best_zc - 1) / best_zc);
    f.blocks = tiles * f.nzch;
    return f;
}

static int device_sms(int device) {
    static int cached[64] = {0};
    if (device < 0 || device >= 64) return 152;
    if (!cached[device]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 152;
        cached[device] = v;
    }
    return cached[device];
}

int fused64_blocks(const Prob* p) { return (int)fused64_grid(p->sys, device_sms(p->ctx->device)).blocks; }

// |w_i| <= ||w||_2 <= ||A v_j||_2 <= ||A||_2 for a unit v_j; Gershgorin
// (with every face term added) bounds ||A||_2.
static double w_bound(const StencilGeom& g, const double* gface) {
    double bound = 4.0 * (fabs(g.kx) + fabs(g.ky) + fabs(g.kz));
    for (int f = 0; f < 6; ++f) bound += fabs(gface[f]);
    return bound > 0.0 ? bound : 1.0;
}

// KV_FUSED64_UNIT=0 in the environment keeps every iteration in the plain
// form (w stored as such): the two forms give the same results to rounding.
static bool unit_form_allowed() {
    static const bool on = [] {
        const char* e = getenv("KV_FUSED64_UNIT");
        return !(e && e[0] == '0');
    }();
    return on;
}

int launch_lanczos_fused64(Prob* p, int j, int it, const void* B, const void* Aprev, void* Wout) {
    const Sys* s = p->sys;
    StencilGeom g;
    g.nx = s->dims[0];
    g.ny = s->ndim >= 2 ? s->dims[1] : 1;
    g.nz = s->ndim >= 3 ? s->dims[2] : 1;
    g.kx = s->coef / (s->h[0] * s->h[0]);
    g.ky = s->ndim >= 2 ? s->coef / (s->h[1] * s->h[1]) : 0.0;
    g.kz = s->ndim >= 3 ? s->coef / (s->h[2] * s->h[2]) : 0.0;
    g.kc = -2.0 * (g.kx + g.ky + g.kz);
    const Fused64Grid f = fused64_grid(s, device_sms(p->ctx->device));
    if (f.blocks < 1 || f.blocks > INT32_MAX) {
        set_error("fused FP64 grid of %lld blocks", (long long)f.blocks);
        return KV_EINVAL;
    }
    CUtensorMap mB, mS;
    int rc = make_grid_map(&mB, const_cast<void*>(B), g.nx, g.ny, g.nz, 8, DBW, DBH);
    if (!rc) rc = make_grid_map(&mS, const_cast<void*>(B), g.nx, g.ny, g.nz, 8, DSW, DBH);
    if (rc) return rc;
    Fused64Args a;
    a.W = (double*)Wout;
    a.Aprev = (const double*)Aprev;
    a.g = g;
    for (int q = 0; q < 6; ++q) {
        a.gface[q] = s->face[q];
        a.gfh[q] = (float)s->face[q];
        a.gfl[q] = (float)(s->face[q] - (double)a.gfh[q]);
        const double kap = q < 2 ? g.kx : (q < 4 ? g.ky : g.kz);
        a.kmg[q] = kap - s->face[q];
        a.kmgx[q] = g.kx > 0.0 ? a.kmg[q] / g.kx : 0.0;
    }
    a.wbound = w_bound(g, s->face);
    // the unit form: kappa_x > 0 and at most 64 bits of drift an iteration
    a.unit_ok = g.kx > 0.0 && 3.0 * a.wbound / g.kx < 0x1p64 && unit_form_allowed();
    a.ry = a.unit_ok ? g.ky / g.kx : 0.0;
    a.rz = a.unit_ok ? g.kz / g.kx : 0.0;
    a.ikx = a.unit_ok ? 1.0 / g.kx : 0.0;
    a.zc = f.zc;
    a.nbx = f.nbx;
    a.nby = f.nby;
    a.st = p->d_state + j;
    a.H = p->d_H + (int64_t)j * (p->m + 1) * p->m;
    a.P = p->d_P + (int64_t)j * p->o * p->m;
    a.cd = CDesc{p->o, p->d_crp, p->d_ccol, p->d_cval, p->N};
    a.m = p->m;
    a.j = it;
    a.red = p->red;
    rc = fused64_prepare();
    if (rc) return rc;
    LaunchScope ls(p->ctx, "lanczos_fused64");
    cudaStream_t st = p->ctx->stream;
    const dim3 grd((unsigned)f.blocks);
    // programmatic dependent launch: the launch and the CTAs' start overlap
    // the previous kernel's last CTA (the grid reduction and the projection)
    const bool pdl = dep_launch_ok(p->ctx);
    auto kern = s->faces ? (it == 0 ? k_lanczos_fused64<true, true> : k_lanczos_fused64<false, true>)
                         : (it == 0 ? k_lanczos_fused64<true, false> : k_lanczos_fused64<false, false>);
    KV_CHECK_CUDA(launch_dep(pdl, kern, grd, dim3(DNT), (size_t)DSMEM_TOTAL, st, mB, mS, a));
    return KV_OK;
}

}  // namespace kv
