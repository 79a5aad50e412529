// Fused fourth-order (2,4) Yee step (H then E in one pass over HBM) for sm_103a.
//
// The update is that of k_fused.cu with every difference of Eq. 2 replaced by the staggered
// fourth-order difference of order4.cuh (taps at +-1/2 and +-3/2, image-closed PEC walls folded
// into per-position weights).  A step reads copy s and writes copy 1-s (ping-pong).
//
// Work: a tile is a 64 x TY column of cells over planes [kz0, kz1); persistent CTAs take their
// tiles and march each one upward in z.  E at plane e needs H^{n+1/2} at planes e-2 .. e+1 (own
// cells) and at plane e with a halo of 2 cells below and 1 above in x and y; H at plane p needs E
// at planes p-1 .. p+2 and, in plane, a halo of 3 below and 2 above.  A "unit" is one plane of the
// six fields (x halo rounded to the 16-byte TMA granule, 3 rows of y halo on either side, one 4-D
// TMA load) plus the material ids; a tile streams the units of planes P0-1 .. PE+2 where
// P0 = max(kz0-2, 0) and PE = kz1, and iteration p = P0 .. PE computes H at plane p and E at
// plane p-1.
//
// Warp roles (TY + 4 warps):
//   * TY row warps: warp w owns row y = w (2 x-adjacent cells per lane); H of its cells, then E one
//     plane behind.  The E values a cell needs across z (Ex, Ey at planes p-1 .. p+2) and the H it
//     computed (Hx, Hy at planes p-3 .. p) live in registers;
//   * 3 halo warps: Hx and Hz on the rows y = -2, -1, TY, and Hy and Hz on the column x = -2, -1
//     or 64 (one lane per row);
//   * producer warp: streams units through an S-slot ring with TMA (full/empty mbarriers), as in
//     k_fused.cu.
// H goes to one of three shared plane buffers (x -2 .. 64, y -2 .. TY), zero at positions outside
// the cavity (the images are in the weights); with three buffers one named barrier per plane
// orders every H write before the E phase that reads it and after the E phase that read the
// buffer's previous plane.  Every wait is bounded (globaltimer); the first to run out raises a
// shared abort flag and the CTA ends as k_fused.cu's does (fdtd_debug_inject_timeout exercises this:
// CTA 0 withholds its first unit and its waits give up after the requested time).
//
// Bytes per cell and step: the 49 B (FP32) / 25 B (16-bit) of the second-order fused kernel; halo
// rows, columns and planes are re-read from L2.
#include "fused_common.cuh"
#include "launch.h"
#include "order4.cuh"

namespace fdtd {

namespace {

using namespace fused;
using namespace o4;

constexpr int TX4 = kTileX;
constexpr int NTR4 = 8;
constexpr uint64_t kWaitLimitNs4 = 2000000000ull;

template <typename T> struct Geom4 {
    static constexpr int HX = 16 / (int)sizeof(T);   // x halo rounded to a 16-byte granule (>= 3 cells)
    static constexpr int BX = TX4 + 2 * HX;           // field box width
    static constexpr int IDX_HALO = 16;               // id box starts 16 bytes left of x0
    static constexpr int IBX = TX4 + 32;              // id box width (bytes): x0-16 .. x0+80
};

struct Fused4Params {
    const TileRec *recs;
    const long long *step;   // batch step clock compared with TileRec::stop (NULL: a single cavity)
    int ntiles;
    int parity;
    int *status;
    int stages;
    int slot_bytes;
    const int *first;   // per-CTA tile ranges (NULL: round-robin)
    int inject_timeout_us;   // >0: CTA 0 never issues its first unit; its waits give up after this many us
};

__host__ __device__ constexpr int al4(int v, int a) { return (v + a - 1) / a * a; }

template <int TY> __host__ __device__ constexpr int box_rows4() { return TY + 6; }
template <typename T, int TY> __host__ __device__ constexpr int field_bytes4() {
    return Geom4<T>::BX * box_rows4<TY>() * (int)sizeof(T);
}
template <int TY> __host__ __device__ constexpr int id_bytes4() { return Geom4<float>::IBX * box_rows4<TY>(); }
template <typename T, int TY> __host__ __device__ constexpr int slot_bytes4() {
    return al4(al4(6 * field_bytes4<T, TY>(), 128) + id_bytes4<TY>(), 128);
}
constexpr int HP4 = TX4 + 4;   // H buffer row pitch: column x + 2 holds x (x = -2 .. 64)
template <int TY> __host__ __device__ constexpr int hrows4() { return TY + 3; }   // y = -2 .. TY
template <int TY> __host__ __device__ constexpr int hbuf_floats4() { return 3 * hrows4<TY>() * HP4; }
constexpr int TAB4_BYTES = kMaxTable * 2 * 16;
template <typename T, int TY> __host__ __device__ constexpr int smem_bytes4(int stages) {
    return 256 + NTR4 * (int)sizeof(TileRec) + TAB4_BYTES + al4(3 * hbuf_floats4<TY>() * 4, 128) +
           stages * slot_bytes4<T, TY>() + 128;
}
template <int TY> __host__ __device__ constexpr int block_threads4() { return (TY + 4) * 32; }

template <typename T, int TY>
__global__ void __launch_bounds__(block_threads4<TY>(), (TY <= 4 ? 2 : 1)) fused4_step_kernel(const Fused4Params P) {
    using G = Geom4<T>;
    constexpr int HX = G::HX, BX = G::BX, IBX = G::IBX;
    constexpr int FB = field_bytes4<T, TY>();
    constexpr int FE = FB / (int)sizeof(T);     // elements per field box (the 4-D box is dense)
    constexpr int NCW = TY + 3;                 // consumer warps
    constexpr int NCT = NCW * 32;
    constexpr int HB = hbuf_floats4<TY>();      // floats per H plane buffer
    constexpr int HC = hrows4<TY>() * HP4;      // floats per component in a buffer
    static_assert(FB % 8 == 0, "field boxes must keep 8-byte alignment");
    static_assert(TY <= 32, "one halo-column cell per lane");

    extern __shared__ __align__(128) unsigned char smem[];
    if (smem_u32(smem) & 127u) {
        if (threadIdx.x == 0) atomicOr(P.status, STATUS_BADINDEX);
        return;
    }
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 8;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 128);
    TileRec *recs = reinterpret_cast<TileRec *>(smem + 256);
    float4 *stab = reinterpret_cast<float4 *>(smem + 256 + NTR4 * sizeof(TileRec));
    float *hbuf = reinterpret_cast<float *>(smem + 256 + NTR4 * sizeof(TileRec) + TAB4_BYTES);
    unsigned char *slots = reinterpret_cast<unsigned char *>(hbuf) + al4(3 * HB * 4, 128);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = P.stages, SB = P.slot_bytes;
    const long long clock = P.step ? *P.step : 0;   // batch step clock: finished members' tiles are skipped
    const int t_begin = P.first ? __ldg(P.first + blockIdx.x) : (int)blockIdx.x;
    const int t_end = P.first ? __ldg(P.first + blockIdx.x + 1) : P.ntiles;
    const int t_step = P.first ? 1 : (int)gridDim.x;
    const bool inject = P.inject_timeout_us > 0 && blockIdx.x == 0;
    const uint64_t lim = inject ? (uint64_t)P.inject_timeout_us * 1000ull : kWaitLimitNs4;

    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        fence_mbarrier_init();
        fence_proxy_async_smem();
    }
    __syncthreads();

    // =========================================================== producer warp
    if (warp == TY + 3) {
        int issued = 0, m = 0, s = 0;
        uint32_t rnd = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; t += t_step) {
            if (__ldg(&P.recs[t].stop) <= clock) continue;   // member already took its last step
            TileRec *rec = &recs[m++ % NTR4];
            int u0 = 0, u1 = 0;   // planes of the tile's first and last unit
            for (int u = 0;; ++u) {
                if (issued >= S) {
                    const bool w = mbar_wait_abortable(&empty[s], rnd ^ 1u, lim, abort_flag, 0);
                    if (!__all_sync(0xffffffffu, w)) {
                        ok = false;
                        break;
                    }
                }
                if (__any_sync(0xffffffffu, *abort_flag != 0)) {
                    ok = false;
                    break;
                }
                if (u == 0) {   // publish the tile record (after the slot wait)
                    const uint32_t *src = reinterpret_cast<const uint32_t *>(P.recs + t);
                    uint32_t *dst = reinterpret_cast<uint32_t *>(rec);
                    for (int q = lane; q < (int)(sizeof(TileRec) / 4); q += 32) dst[q] = __ldg(src + q);
                    __syncwarp();
                    u0 = (rec->kz0 > 2 ? rec->kz0 - 2 : 0) - 1;
                    u1 = rec->kz1 + 2;
                }
                const int kk = u0 + u;
                if (lane == 0 && !(inject && issued == 0)) {
                    const int src_copy = P.parity ^ rec->parity_off;
                    const bool has_id = rec->mode == COEF_ID8;
                    unsigned char *dst = slots + s * SB;
                    fence_proxy_async_smem();
                    if (tma_x_ok(P.status, rec->x0 - HX, (int)sizeof(T)) &&
                        (!has_id || tma_x_ok(P.status, rec->x0 - G::IDX_HALO, 1))) {
                        mbar_arrive_expect_tx(&full[s], 6 * FB + (has_id ? id_bytes4<TY>() : 0));
                        tma_load_4d(dst, rec->maps + src_copy * 6, rec->x0 - HX, rec->y0 - 3, kk, 0, &full[s]);
                        if (has_id)
                            tma_load_3d(dst + al4(6 * FB, 128), rec->maps + 12, rec->x0 - G::IDX_HALO, rec->y0 - 3,
                                        kk, &full[s]);
                    } else {
                        mbar_arrive(&full[s]);   // checked build: the unit is skipped, the slot still completes
                    }
                }
                __syncwarp();
                ++issued;
                if (++s == S) {
                    s = 0;
                    rnd ^= 1u;
                }
                if (kk >= u1) break;
            }
        }
        if (!ok && lane == 0) {
            atomicOr(P.status, STATUS_TIMEOUT);
            for (int u = issued > S ? issued - S : 0; u < issued; ++u) {
                if (inject && u == 0) continue;   // never issued
                mbar_wait_bounded(&full[u % S], (u / S) & 1, kWaitLimitNs4);
            }
        }
        return;
    }

    // =========================================================== consumer warps
    const bool row_warp = warp < TY;
    const int hw = warp - TY;                          // halo warp 0..2 (rows -2, -1, TY; columns -2, -1, 64)
    const int y = row_warp ? warp : (hw == 2 ? TY : hw - 2);
    const int x = 2 * lane;
    const int bxo = x + HX, byo = y + 3;               // the lane's first cell in a field box
    const int xc = hw == 0 ? -2 : hw == 1 ? -1 : TX4;  // halo column of a halo warp
    const bool col_lane = !row_warp && lane < TY;      // lane holds the column cell of row `lane`
    int ws = 0, rs = 0, hb = 0, m = 0;                 // wait cursor, release cursor, H buffer of plane p
    uint32_t wpar = 0;
    const float4 *tab_cached = nullptr;
    auto slot = [&](int s) { return reinterpret_cast<const T *>(slots + s * SB); };
    auto ids_of = [&](int s) { return slots + s * SB + al4(6 * FB, 128); };
    auto at = [&](const T *base, int f, int bx, int by) { return base + f * FE + by * BX + bx; };
    auto wait_next = [&]() -> const T * {
        const bool ok = mbar_wait_abortable(&full[ws], wpar, lim, abort_flag, 0);
        const T *r = ok ? slot(ws) : nullptr;
        if (++ws == S) {
            ws = 0;
            wpar ^= 1u;
        }
        return r;
    };
    auto release = [&]() {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[rs]);
        if (++rs == S) rs = 0;
    };

    for (int t = t_begin; t < t_end; t += t_step) {
        if (__ldg(&P.recs[t].stop) <= clock) continue;   // same skip rule as the producer
        // ---------------- tile start: record, table, prologue units P0-1 .. P0+1 (E z-taps)
        const T *u_a = wait_next();
        if (bar_sync_or(2, NCT, u_a == nullptr || *abort_flag != 0)) {
            if (threadIdx.x == 0) atomicOr(P.status, STATUS_TIMEOUT);
            return;
        }
        const TileRec *rec = &recs[m++ % NTR4];
        const int x0 = rec->x0, y0 = rec->y0, kz0 = rec->kz0, kz1 = rec->kz1;
        const int nx = rec->nx, ny = rec->ny, nz = rec->nz;
        const long long pitch = rec->pitch, plane = rec->plane;
        const bool id_mode = rec->mode == COEF_ID8;
        const bool ch_uni = rec->ch_uniform != 0;
        if (id_mode && rec->table != tab_cached) {
            const float4 *src = rec->table;
            const int n = 2 * rec->ntab;
            for (int e = threadIdx.x; e < n; e += NCT) stab[e] = __ldg(src + e);
            bar_sync_or(2, NCT, false);
            tab_cached = src;
        }
        const float4 *table = stab;
        const int dstc = (P.parity ^ rec->parity_off) ^ 1;
        // the six arrays of a copy lie in one allocation, plane * nz elements apart
        T *const dst0 = static_cast<T *>(rec->dst[dstc][0]);
        const long long fstride = plane * nz;
        const float ce_s0 = rec->ce[0], ce_s1 = rec->ce[1], ce_s2 = rec->ce[2];
        const float ch_s0 = rec->ch[0], ch_s1 = rec->ch[1], ch_s2 = rec->ch[2];
        const int gj = y0 + y, gi = x0 + x;
        const int P0 = kz0 > 2 ? kz0 - 2 : 0, PE = kz1;

        // per-position weights (x per cell, y per row); validity of H at the lane's positions
        const float2 wax_h = make_float2(wa_h(gi, nx), wa_h(gi + 1, nx)), wbx_h = make_float2(wb_h(gi, nx), wb_h(gi + 1, nx));
        const float2 wax_e = make_float2(wa_e(gi, nx), wa_e(gi + 1, nx)), wbx_e = make_float2(wb_e(gi, nx), wb_e(gi + 1, nx));
        const float way_h = wa_h(gj, ny), wby_h = wb_h(gj, ny), way_e = wa_e(gj, ny), wby_e = wb_e(gj, ny);
        const bool vrow = gj >= 0 && gj < ny, v0 = gi < nx, v1 = gi + 1 < nx;
        // halo column cell (row `lane`)
        const int cgy = y0 + lane, cgx = x0 + xc;
        const bool cvalid = col_lane && cgy < ny && cgx >= 0 && cgx < nx;
        const int cbx = xc + HX, cby = lane + 3;

        // z windows: E at planes p-1, p, p+1 (own cells / halo row: Ex, Ey; halo column: Ex);
        // H of own cells at planes p-3, p-2, p-1 (planes below 0 are images: 0)
        float2 hxw0 = make_float2(0.f, 0.f), hxw1 = hxw0, hxw2 = hxw0, hyw0 = hxw0, hyw1 = hxw0, hyw2 = hxw0;
        float2 exw0 = hxw0, exw1 = hxw0, exw2 = hxw0, eyw0 = hxw0, eyw1 = hxw0, eyw2 = hxw0;
        float exc0 = 0.f, exc1 = 0.f, exc2 = 0.f;
        float2 ez_prev = hxw0;
        uint32_t id_prev = 0;
        {
            const T *u_b = wait_next();
            const T *u_c = wait_next();
            const bool ok = u_b && u_c;
            if (ok) {
                exw0 = Pair<T>::ld(at(u_a, 0, bxo, byo));
                exw1 = Pair<T>::ld(at(u_b, 0, bxo, byo));
                exw2 = Pair<T>::ld(at(u_c, 0, bxo, byo));
                eyw0 = Pair<T>::ld(at(u_a, 1, bxo, byo));
                eyw1 = Pair<T>::ld(at(u_b, 1, bxo, byo));
                eyw2 = Pair<T>::ld(at(u_c, 1, bxo, byo));
                if (col_lane) {
                    exc0 = Pair<T>::ld1(at(u_a, 0, cbx, cby));
                    exc1 = Pair<T>::ld1(at(u_b, 0, cbx, cby));
                    exc2 = Pair<T>::ld1(at(u_c, 0, cbx, cby));
                }
            }
            release();   // unit P0 - 1 is read only for its z-taps
        }

#pragma unroll 2   // consecutive planes renamed instead of copied (the z windows): 2.6 % faster
        for (int p = P0; p <= PE; ++p) {
            const T *V = wait_next();            // unit p + 2
            const T *U = slot(rs);               // unit p (landed two iterations ago)
            const unsigned char *ida = ids_of(rs);
            const bool ok = V != nullptr && *abort_flag == 0;
            const bool hcomp = ok && p < nz;
            float *hn = hbuf + hb * HB;
            const float waz_h = wa_h(p, nz), wbz_h = wb_h(p, nz);
            float2 hx_n = make_float2(0.f, 0.f), hy_n = hx_n, ez_cur = hx_n;
            uint32_t id_cur = 0;
            float2 ex3 = hx_n, ey3 = hx_n;
            float exc3 = 0.f;
            if (ok) {
                ex3 = Pair<T>::ld(at(V, 0, bxo, byo));
                ey3 = Pair<T>::ld(at(V, 1, bxo, byo));
                if (col_lane) exc3 = Pair<T>::ld1(at(V, 0, cbx, cby));
            }
            auto ch_at = [&](int bx_id, int by_id, float &cx, float &cy, float &cz) {   // ch of one cell
                cx = ch_s0;
                cy = ch_s1;
                cz = ch_s2;
                if (id_mode && !ch_uni) {
                    const float4 a = table[2 * ida[by_id * IBX + bx_id] + 1];
                    cx = a.x;
                    cy = a.y;
                    cz = a.z;
                }
            };

            // ---------------- phase A: H^{n+1/2} at plane p
            if (hcomp) {
                const float2 wz_a = make_float2(waz_h, waz_h), wz_b = make_float2(wbz_h, wbz_h);
                const float2 wy_a = make_float2(way_h, way_h), wy_b = make_float2(wby_h, wby_h);
                if (row_warp) {
                    const float2 ez_m1 = Pair<T>::ld(at(U, 2, bxo, byo - 1)), ez_0 = Pair<T>::ld(at(U, 2, bxo, byo));
                    const float2 ez_p1 = Pair<T>::ld(at(U, 2, bxo, byo + 1)), ez_p2 = Pair<T>::ld(at(U, 2, bxo, byo + 2));
                    const float ez_l = Pair<T>::ld1(at(U, 2, bxo - 1, byo));
                    const float2 ez_r = Pair<T>::ld(at(U, 2, bxo + 2, byo));
                    const float2 ex_m1 = Pair<T>::ld(at(U, 0, bxo, byo - 1)), ex_p1 = Pair<T>::ld(at(U, 0, bxo, byo + 1));
                    const float2 ex_p2 = Pair<T>::ld(at(U, 0, bxo, byo + 2));
                    const float ey_l = Pair<T>::ld1(at(U, 1, bxo - 1, byo));
                    const float2 ey_r = Pair<T>::ld(at(U, 1, bxo + 2, byo));
                    float2 hx = Pair<T>::ld(at(U, 3, bxo, byo)), hy = Pair<T>::ld(at(U, 4, bxo, byo));
                    float2 hz = Pair<T>::ld(at(U, 5, bxo, byo));
                    float2 chx = make_float2(ch_s0, ch_s0), chy = make_float2(ch_s1, ch_s1), chz = make_float2(ch_s2, ch_s2);
                    if (id_mode) {
                        id_cur = *reinterpret_cast<const uint16_t *>(ida + byo * IBX + x + G::IDX_HALO);
                        if (!ch_uni) {
                            const float4 a = table[2 * (id_cur & 0xff) + 1], b = table[2 * (id_cur >> 8) + 1];
                            chx = make_float2(a.x, b.x);
                            chy = make_float2(a.y, b.y);
                            chz = make_float2(a.z, b.z);
                        }
                    }
                    const float2 dzEy = d4(eyw0, eyw1, eyw2, ey3, wz_a, wz_b);
                    const float2 dzEx = d4(exw0, exw1, exw2, ex3, wz_a, wz_b);
                    const float2 dyEz = d4(ez_m1, ez_0, ez_p1, ez_p2, wy_a, wy_b);
                    const float2 dyEx = d4(ex_m1, exw1, ex_p1, ex_p2, wy_a, wy_b);
                    const float2 dxEz = d4(make_float2(ez_l, ez_0.x), ez_0, make_float2(ez_0.y, ez_r.x), ez_r, wax_h, wbx_h);
                    const float2 dxEy = d4(make_float2(ey_l, eyw1.x), eyw1, make_float2(eyw1.y, ey_r.x), ey_r, wax_h, wbx_h);
                    // each bracket is -(curl E): H + ch * bracket
                    hx = fma2o(chx, sub2o(dzEy, dyEz), hx);
                    hy = fma2o(chy, sub2o(dxEz, dzEx), hy);
                    hz = fma2o(chz, sub2o(dyEx, dxEy), hz);
                    const bool a0 = vrow && v0, a1 = vrow && v1;
                    hx = make_float2(a0 ? hx.x : 0.f, a1 ? hx.y : 0.f);
                    hy = make_float2(a0 ? hy.x : 0.f, a1 ? hy.y : 0.f);
                    hz = make_float2(a0 ? hz.x : 0.f, a1 ? hz.y : 0.f);
                    const int o = (y + 2) * HP4 + x + 2;
                    *reinterpret_cast<float2 *>(hn + o) = hx;
                    *reinterpret_cast<float2 *>(hn + HC + o) = hy;
                    *reinterpret_cast<float2 *>(hn + 2 * HC + o) = hz;
                    const long long g = (long long)p * plane + (long long)gj * pitch + gi;
                    if (p >= kz0 && p < kz1 && a0 && store_ok(P.status, g, 2, plane * nz)) {
                        Pair<T>::st_cs(dst0 + g + 3 * fstride, hx.x, hx.y);
                        Pair<T>::st_cs(dst0 + g + 4 * fstride, hy.x, hy.y);
                        Pair<T>::st_cs(dst0 + g + 5 * fstride, hz.x, hz.y);
                    }
                    hx_n = hx;
                    hy_n = hy;
                    ez_cur = ez_0;
                } else {
                    // halo row y: Hx and Hz on the lane's two cells
                    const float2 ez_m1 = Pair<T>::ld(at(U, 2, bxo, byo - 1)), ez_0 = Pair<T>::ld(at(U, 2, bxo, byo));
                    const float2 ez_p1 = Pair<T>::ld(at(U, 2, bxo, byo + 1)), ez_p2 = Pair<T>::ld(at(U, 2, bxo, byo + 2));
                    const float2 ex_m1 = Pair<T>::ld(at(U, 0, bxo, byo - 1)), ex_0 = Pair<T>::ld(at(U, 0, bxo, byo));
                    const float2 ex_p1 = Pair<T>::ld(at(U, 0, bxo, byo + 1)), ex_p2 = Pair<T>::ld(at(U, 0, bxo, byo + 2));
                    const float ey_l = Pair<T>::ld1(at(U, 1, bxo - 1, byo));
                    const float2 ey_r = Pair<T>::ld(at(U, 1, bxo + 2, byo));
                    float2 hx = Pair<T>::ld(at(U, 3, bxo, byo)), hz = Pair<T>::ld(at(U, 5, bxo, byo));
                    float2 chx = make_float2(ch_s0, ch_s0), chz = make_float2(ch_s2, ch_s2);
                    if (id_mode && !ch_uni) {
                        const uint32_t ip = *reinterpret_cast<const uint16_t *>(ida + byo * IBX + x + G::IDX_HALO);
                        const float4 a = table[2 * (ip & 0xff) + 1], b = table[2 * (ip >> 8) + 1];
                        chx = make_float2(a.x, b.x);
                        chz = make_float2(a.z, b.z);
                    }
                    const float2 dzEy = d4(eyw0, eyw1, eyw2, ey3, wz_a, wz_b);
                    const float2 dyEz = d4(ez_m1, ez_0, ez_p1, ez_p2, wy_a, wy_b);
                    const float2 dyEx = d4(ex_m1, ex_0, ex_p1, ex_p2, wy_a, wy_b);
                    const float2 dxEy = d4(make_float2(ey_l, eyw1.x), eyw1, make_float2(eyw1.y, ey_r.x), ey_r, wax_h, wbx_h);
                    hx = fma2o(chx, sub2o(dzEy, dyEz), hx);
                    hz = fma2o(chz, sub2o(dyEx, dxEy), hz);
                    const bool a0 = vrow && v0, a1 = vrow && v1;
                    const int o = (y + 2) * HP4 + x + 2;
                    *reinterpret_cast<float2 *>(hn + o) = make_float2(a0 ? hx.x : 0.f, a1 ? hx.y : 0.f);
                    *reinterpret_cast<float2 *>(hn + 2 * HC + o) = make_float2(a0 ? hz.x : 0.f, a1 ? hz.y : 0.f);
                    if (col_lane) {
                        // halo column x = xc of row `lane`: Hy and Hz
                        auto E1 = [&](int f, int dx_, int dy_) { return Pair<T>::ld1(at(U, f, cbx + dx_, cby + dy_)); };
                        float cchx, cchy, cchz;
                        ch_at(xc + G::IDX_HALO, cby, cchx, cchy, cchz);
                        const float cwax = wa_h(cgx, nx), cwbx = wb_h(cgx, nx);
                        const float cway = wa_h(cgy, ny), cwby = wb_h(cgy, ny);
                        const float dxEz_c = d4(E1(2, -1, 0), E1(2, 0, 0), E1(2, 1, 0), E1(2, 2, 0), cwax, cwbx);
                        const float dzEx_c = d4(exc0, exc1, exc2, exc3, waz_h, wbz_h);
                        const float dyEx_c = d4(E1(0, 0, -1), exc1, E1(0, 0, 1), E1(0, 0, 2), cway, cwby);
                        const float dxEy_c = d4(E1(1, -1, 0), E1(1, 0, 0), E1(1, 1, 0), E1(1, 2, 0), cwax, cwbx);
                        const float chy_ = __fmaf_rn(cchy, __fsub_rn(dxEz_c, dzEx_c), E1(4, 0, 0));
                        const float chz_ = __fmaf_rn(cchz, __fsub_rn(dyEx_c, dxEy_c), E1(5, 0, 0));
                        const int oc = (lane + 2) * HP4 + xc + 2;
                        hn[HC + oc] = cvalid ? chy_ : 0.f;
                        hn[2 * HC + oc] = cvalid ? chz_ : 0.f;
                    }
                }
            }
            release();   // unit p
            // all of plane p's H (own cells, halo rows and columns) is in buffer hb from here on, and
            // every warp is past the E phase that read the buffer hb + 1 (mod 3) last
            asm volatile("bar.sync 1, %0;" ::"r"(NCT) : "memory");

            // ---------------- phase B: E^{n+1} at plane e = p - 1 (row warps)
            const int e = p - 1;
            if (row_warp && ok && e >= kz0 && e < kz1) {
                const float *hq = hbuf + (hb == 0 ? 2 : hb - 1) * HB;   // plane e
                const int o = (y + 2) * HP4 + x + 2;
                const float2 hz_m2 = *reinterpret_cast<const float2 *>(hq + 2 * HC + o - 2 * HP4);
                const float2 hz_m1 = *reinterpret_cast<const float2 *>(hq + 2 * HC + o - HP4);
                const float2 hz_0 = *reinterpret_cast<const float2 *>(hq + 2 * HC + o);
                const float2 hz_p1 = *reinterpret_cast<const float2 *>(hq + 2 * HC + o + HP4);
                const float2 hz_l = *reinterpret_cast<const float2 *>(hq + 2 * HC + o - 2);
                const float hz_r = hq[2 * HC + o + 2];
                const float2 hy_l = *reinterpret_cast<const float2 *>(hq + HC + o - 2);
                const float hy_r = hq[HC + o + 2];
                const float2 hx_m2 = *reinterpret_cast<const float2 *>(hq + o - 2 * HP4);
                const float2 hx_m1 = *reinterpret_cast<const float2 *>(hq + o - HP4);
                const float2 hx_p1 = *reinterpret_cast<const float2 *>(hq + o + HP4);
                float4 ce_a = make_float4(ce_s0, ce_s1, ce_s2, 0.f), ce_b = ce_a;
                if (id_mode) {
                    ce_a = table[2 * (id_prev & 0xff)];
                    ce_b = table[2 * (id_prev >> 8)];
                }
                // PEC: a zero coefficient leaves a tangential E exactly unchanged
                const bool k1 = e >= 1, j1 = gj >= 1, i1 = gi >= 1;
                const float2 cex = (j1 && k1) ? make_float2(ce_a.x, ce_b.x) : make_float2(0.f, 0.f);
                const float2 cey = make_float2((i1 && k1) ? ce_a.y : 0.f, k1 ? ce_b.y : 0.f);
                const float2 cez = make_float2((i1 && j1) ? ce_a.z : 0.f, j1 ? ce_b.z : 0.f);
                const float wze_a = wa_e(e, nz), wze_b = wb_e(e, nz);
                const float2 wz_a = make_float2(wze_a, wze_a), wz_b = make_float2(wze_b, wze_b);
                const float2 wy_a = make_float2(way_e, way_e), wy_b = make_float2(wby_e, wby_e);
                const float2 dyHz = d4(hz_m2, hz_m1, hz_0, hz_p1, wy_a, wy_b);
                const float2 dzHy = d4(hyw0, hyw1, hyw2, hy_n, wz_a, wz_b);
                const float2 dzHx = d4(hxw0, hxw1, hxw2, hx_n, wz_a, wz_b);
                const float2 dxHz = d4(hz_l, make_float2(hz_l.y, hz_0.x), hz_0, make_float2(hz_0.y, hz_r), wax_e, wbx_e);
                const float2 dxHy = d4(hy_l, make_float2(hy_l.y, hyw2.x), hyw2, make_float2(hyw2.y, hy_r), wax_e, wbx_e);
                const float2 dyHx = d4(hx_m2, hx_m1, hxw2, hx_p1, wy_a, wy_b);
                const float2 ex = fma2o(cex, sub2o(dyHz, dzHy), exw0);
                const float2 ey = fma2o(cey, sub2o(dzHx, dxHz), eyw0);
                const float2 ez = fma2o(cez, sub2o(dxHy, dyHx), ez_prev);
                const long long g = (long long)e * plane + (long long)gj * pitch + gi;
                if (gj < ny && gi < nx && store_ok(P.status, g, 2, plane * nz)) {
                    Pair<T>::st_cs(dst0 + g, ex.x, ex.y);
                    Pair<T>::st_cs(dst0 + g + 1 * fstride, ey.x, ey.y);
                    Pair<T>::st_cs(dst0 + g + 2 * fstride, ez.x, ez.y);
                }
            }
            // ---------------- slide the z windows
            exw0 = exw1; exw1 = exw2; exw2 = ex3;
            eyw0 = eyw1; eyw1 = eyw2; eyw2 = ey3;
            exc0 = exc1; exc1 = exc2; exc2 = exc3;
            hxw0 = hxw1; hxw1 = hxw2; hxw2 = hx_n;
            hyw0 = hyw1; hyw1 = hyw2; hyw2 = hy_n;
            ez_prev = ez_cur;
            id_prev = id_cur;
            hb = hb == 2 ? 0 : hb + 1;
        }
        // units PE + 1 and PE + 2 were read for their z-taps only
        release();
        release();
    }
}

template <typename T, int TY>
cudaError_t launch4_typed(const FusedLaunch &L, cudaStream_t s) {
    const int smem = smem_bytes4<T, TY>(L.stages);
    auto kern = fused4_step_kernel<T, TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    Fused4Params P;
    P.recs = L.recs;
    P.step = L.step;
    P.ntiles = L.ntiles;
    P.parity = L.parity;
    P.status = L.status;
    P.stages = L.stages;
    P.slot_bytes = slot_bytes4<T, TY>();
    P.first = L.first;
    P.inject_timeout_us = L.inject_timeout_us;
    kern<<<L.grid, block_threads4<TY>(), smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T, int TY>
cudaError_t occupancy4_typed(int stages, int *n) {
    const int smem = smem_bytes4<T, TY>(stages);
    auto kern = fused4_step_kernel<T, TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, block_threads4<TY>(), smem);
}

#define FDTD4_DISPATCH(storage, tile_y, ...)                                                       \
    do {                                                                                           \
        if (storage == 0) {                                                                        \
            if (tile_y == 4) { using T = float; constexpr int TY = 4; __VA_ARGS__; }               \
            else if (tile_y == 8) { using T = float; constexpr int TY = 8; __VA_ARGS__; }          \
            else if (tile_y == 12) { using T = float; constexpr int TY = 12; __VA_ARGS__; }          \
            else if (tile_y == 16) { using T = float; constexpr int TY = 16; __VA_ARGS__; }        \
        } else if (storage == 1) {                                                                 \
            if (tile_y == 4) { using T = __half; constexpr int TY = 4; __VA_ARGS__; }              \
            else if (tile_y == 8) { using T = __half; constexpr int TY = 8; __VA_ARGS__; }         \
            else if (tile_y == 12) { using T = __half; constexpr int TY = 12; __VA_ARGS__; }         \
            else if (tile_y == 16) { using T = __half; constexpr int TY = 16; __VA_ARGS__; }       \
        } else if (storage == 2) {                                                                 \
            if (tile_y == 4) { using T = __nv_bfloat16; constexpr int TY = 4; __VA_ARGS__; }       \
            else if (tile_y == 8) { using T = __nv_bfloat16; constexpr int TY = 8; __VA_ARGS__; }  \
            else if (tile_y == 12) { using T = __nv_bfloat16; constexpr int TY = 12; __VA_ARGS__; }  \
            else if (tile_y == 16) { using T = __nv_bfloat16; constexpr int TY = 16; __VA_ARGS__; } \
        }                                                                                          \
    } while (0)

}  // namespace

int fused4_smem_bytes(int storage, int tile_y, int stages) {
    int r = -1;
    FDTD4_DISPATCH(storage, tile_y, r = smem_bytes4<T, TY>(stages));
    return r;
}

cudaError_t fused4_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm) {
    cudaError_t e = cudaErrorInvalidValue;
    FDTD4_DISPATCH(storage, tile_y, e = occupancy4_typed<T, TY>(stages, ctas_per_sm));
    return e;
}

cudaError_t launch_fused4_step(int storage, const FusedLaunch &L, cudaStream_t s) {
    if (L.ntiles <= 0) return cudaSuccess;
    if (L.stages < 4 || L.stages > 8) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    FDTD4_DISPATCH(storage, L.tile_y, e = launch4_typed<T, TY>(L, s));
    return e;
}

}  // namespace fdtd
