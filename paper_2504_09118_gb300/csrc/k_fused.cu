// Fused Yee step (H then E in one pass over HBM) for sm_103a.
//
// The update is Eq. 2 of the paper in the order of Listing 1: H^{n+1/2} from
// curl E^n, then E^{n+1} from curl H^{n+1/2}; PEC by index predicates
// (tangential E is never updated, normal H on a face sees a zero curl).  A
// step reads copy s of the six fields and writes copy 1-s (ping-pong), so a
// tile recomputes the H values on its lower x/y halo from unmodified E rather
// than waiting for the neighbouring tile.
//
// Work: a tile is a 64 x TY column of cells over planes [kz0, kz1); persistent
// CTAs take tiles round-robin and march each one upward in z.  Plane k needs
// "unit" k (six fields + material id at plane k, one-cell halo in x and y,
// the x halo widened to the 16-byte TMA granule) and unit k+1 (E at k+1 for
// the z derivative of H).
//
// Warp roles (TY + 2 warps):
//   * producer warp: walks the CTA's tiles, copies each tile's record (host
//     built: origin, extents, pointers, scales, coefficients) into a small
//     shared ring, and streams units into an S-slot ring with 3-D TMA loads
//     (full[s] mbarrier: expect_tx + complete_tx), gated by empty[s];
//   * TY row warps: warp w owns row y = w: it computes H on 2 x-adjacent cells
//     per lane (64 cells), keeps them and the loaded E in registers, publishes
//     H to a double-buffered shared plane, and after one named barrier updates
//     E on the same cells; H^{n+1/2}(k-1) of its cells stays in registers for
//     the z derivative of the next plane;
//   * halo warp: H on the row y = -1 (Hx, Hz) and the column x = -1 (Hy, Hz),
//     needed by the E update of the tile's first row and column; phase A only.
// One plain named barrier per plane; a consumer warp releases a unit (arrive
// on empty[s]) once it no longer reads it.  Arithmetic uses the packed FP32x2
// instructions of sm_100+ over each lane's two cells.
//
// Bytes per cell and plane: 6 loads + 6 stores of the storage type + one
// material-id byte (49 B in FP32, 25 B in 16-bit storage); halo rows are
// re-read from L2.  Every mbarrier wait is bounded in wall time (globaltimer):
// the first wait that runs out raises a shared abort flag, after which every
// wait returns at once; the consumers leave together at the next tile start
// (an OR-reducing barrier) after latching STATUS_TIMEOUT, and the producer
// stops issuing, drains its in-flight copies (bounded again) and exits.
#include "fused_common.cuh"
#include "launch.h"

namespace fdtd {

namespace {

using namespace fused;

#ifndef FDTD_PRODUCER_SLEEP_NS
#define FDTD_PRODUCER_SLEEP_NS 0   // back-off of the producer warp between polls of a full ring slot
#endif

constexpr int TX = kTileX;
constexpr int NTR = 8;                              // tile-record ring entries
constexpr uint64_t kWaitLimitNs = 2000000000ull;    // 2 s: far beyond any healthy TMA latency

template <typename T> struct FusedGeom {
    static constexpr int HX = 16 / (int)sizeof(T);  // x halo rounded to a 16-byte TMA granule
    static constexpr int BX = TX + 2 * HX;          // field box width (elements)
    static constexpr int IDX_HALO = 16;             // id box starts 16 bytes left of x0
    static constexpr int IBX = TX + IDX_HALO;       // id box width (bytes)
};

struct FusedParams {
    const TileRec *recs;
    const long long *step;
    int ntiles;
    int parity;
    int *status;
    int stages;
    int slot_bytes;
    int inject_timeout_us;
    const int *first;   // per-CTA tile ranges (NULL: round-robin)
};

__host__ __device__ constexpr int align_up(int v, int a) { return (v + a - 1) / a * a; }

template <typename T, int TY>
__host__ __device__ constexpr int field_box_bytes() {
    return FusedGeom<T>::BX * (TY + 2) * (int)sizeof(T);
}
template <int TY>
__host__ __device__ constexpr int id_box_bytes() {
    return FusedGeom<float>::IBX * (TY + 2);
}
template <typename T, int TY>
__host__ __device__ constexpr int field_box_stride() {   // each TMA destination on a 128-byte boundary
    return align_up(field_box_bytes<T, TY>(), 128);
}
template <typename T, int TY>
__host__ __device__ constexpr int slot_bytes() {
    return align_up(6 * field_box_stride<T, TY>() + id_box_bytes<TY>(), 128);
}
constexpr int HP = TX + 2;   // shared H plane row pitch; column x + 2 holds x (x = -1 .. TX-1)
template <int TY>
__host__ __device__ constexpr int hbuf_floats() {
    return 3 * (TY + 1) * HP;
}
constexpr int TAB_BYTES = kMaxTable * 2 * 16;   // shared copy of a cavity's material table (ce, ch float4)
template <typename T, int TY>
__host__ __device__ constexpr int smem_bytes(int stages) {
    return 256 /*barriers, abort flag*/ + NTR * (int)sizeof(TileRec) + TAB_BYTES + align_up(2 * hbuf_floats<TY>() * 4, 128) +
           stages * slot_bytes<T, TY>() + 128 /*alignment slack*/;
}
template <int TY>
__host__ __device__ constexpr int block_threads() {
    return (TY + 2) * 32;
}

template <typename T, int TY>
__global__ void __launch_bounds__(block_threads<TY>(), (TY <= 8 ? 2 : 1)) fused_step_kernel(const FusedParams P) {
    using G = FusedGeom<T>;
    constexpr int HX = G::HX, BX = G::BX;
    constexpr int FB = field_box_bytes<T, TY>();
    constexpr int FS = field_box_stride<T, TY>();
    constexpr int FE = FS / (int)sizeof(T);
    constexpr int NCW = TY + 1;                 // consumer warps: TY row warps + halo warp
    constexpr int NCT = NCW * 32;
    constexpr int HB = hbuf_floats<TY>();       // floats per H plane buffer
    constexpr int HC = (TY + 1) * HP;           // floats per component in a buffer

    // Indexed directly (no pointer round trip through an integer) so that every access keeps the
    // shared-memory address space.  The dynamic region starts on a 1 KiB boundary when the kernel
    // declares no static shared memory; the check below turns any other layout into an error.
    extern __shared__ __align__(128) unsigned char smem[];
    if (smem_u32(smem) & 127u) {
        if (threadIdx.x == 0) atomicOr(P.status, STATUS_BADINDEX);
        return;
    }
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 8;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 128);   // set by the first wait that runs out
    TileRec *recs = reinterpret_cast<TileRec *>(smem + 256);
    float4 *stab = reinterpret_cast<float4 *>(smem + 256 + NTR * sizeof(TileRec));
    float *hbuf = reinterpret_cast<float *>(smem + 256 + NTR * sizeof(TileRec) + TAB_BYTES);
    unsigned char *slots = reinterpret_cast<unsigned char *>(hbuf) + align_up(2 * HB * 4, 128);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = P.stages, SB = P.slot_bytes;
    const long long step = P.step ? *P.step : 0;   // launch index within a batch
    // this CTA's tiles: a host-balanced contiguous range, or every gridDim.x-th tile
    const int t_begin = P.first ? __ldg(P.first + blockIdx.x) : (int)blockIdx.x;
    const int t_end = P.first ? __ldg(P.first + blockIdx.x + 1) : P.ntiles;
    const int t_step = P.first ? 1 : (int)gridDim.x;
    const bool inject = P.inject_timeout_us > 0 && blockIdx.x == 0;
    const uint64_t lim = inject ? (uint64_t)P.inject_timeout_us * 1000ull : kWaitLimitNs;

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
    if (warp == TY + 1) {
        int issued = 0, m = 0;
        int s = 0;           // slot of the next unit
        uint32_t rnd = 0;    // parity of the ring round of the next unit
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; t += t_step) {
            if (__ldg(&P.recs[t].stop) <= step) continue;   // member already took its last step
            TileRec *rec = &recs[m++ % NTR];
            int kb = 0, kz1 = 0;
            for (int k = 0;; ++k) {
                if (issued >= S) {   // wait until unit issued - S (same slot, previous round) is released
                    const bool w = mbar_wait_abortable(&empty[s], rnd ^ 1u, lim, abort_flag, FDTD_PRODUCER_SLEEP_NS);
                    if (!__all_sync(0xffffffffu, w)) {
                        ok = false;
                        break;
                    }
                }
                if (__any_sync(0xffffffffu, *abort_flag != 0)) {
                    ok = false;
                    break;
                }
                if (k == 0) {   // first unit of the tile: publish the tile record (after the slot wait)
                    const uint32_t *src = reinterpret_cast<const uint32_t *>(P.recs + t);
                    uint32_t *dst = reinterpret_cast<uint32_t *>(rec);
                    for (int q = lane; q < (int)(sizeof(TileRec) / 4); q += 32) dst[q] = __ldg(src + q);
                    __syncwarp();
                    kb = rec->kz0 > 0 ? rec->kz0 - 1 : rec->kz0;
                    kz1 = rec->kz1;
                }
                const int kk = kb + k;
                if (lane == 0 && !(inject && issued == 0)) {
                    const int src_copy = P.parity ^ rec->parity_off;
                    const bool has_id = rec->mode == COEF_ID8;
                    unsigned char *dst = slots + s * SB;
                    fence_proxy_async_smem();
                    if (tma_x_ok(P.status, rec->x0 - HX, (int)sizeof(T)) &&
                        (!has_id || tma_x_ok(P.status, rec->x0 - G::IDX_HALO, 1))) {
                        mbar_arrive_expect_tx(&full[s], 6 * FB + (has_id ? id_box_bytes<TY>() : 0));
                        const CUtensorMap *mp = rec->maps + src_copy * 6;
#pragma unroll
                        for (int f = 0; f < 6; ++f)
                            tma_load_3d(dst + f * FS, mp + f, rec->x0 - HX, rec->y0 - 1, kk, &full[s]);
                        if (has_id)
                            tma_load_3d(dst + 6 * FS, rec->maps + 12, rec->x0 - G::IDX_HALO, rec->y0 - 1, kk,
                                        &full[s]);
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
                if (kk >= kz1) break;
            }
        }
        if (!ok && lane == 0) {
            atomicOr(P.status, STATUS_TIMEOUT);
            // drain this CTA's copies still in flight before its shared memory goes away
            for (int u = issued > S ? issued - S : 0; u < issued; ++u) {
                if (inject && u == 0) continue;
                mbar_wait_bounded(&full[u % S], (u / S) & 1, kWaitLimitNs);
            }
        }
        return;
    }

    // =========================================================== consumer warps
    const bool halo = warp == TY;
    const int y = halo ? -1 : warp;             // row of this warp (tile-local)
    const int x = 2 * lane;                     // first of the lane's two cells
    const int bx = x + HX, by = y + 1;          // position in a field box
    int sa = 0, m = 0, hb = 0;                  // slot of the current unit, tile count, H buffer
    uint32_t pa = 0;                            // phase parity of that slot
    const float4 *tab_cached = nullptr;
    float2 hpx = make_float2(0.f, 0.f), hpy = make_float2(0.f, 0.f);   // H^{n+1/2}(k-1) of own cells
    auto wait_full = [&](int slot, uint32_t par) { return mbar_wait_abortable(&full[slot], par, lim, abort_flag, 0); };

    for (int t = t_begin; t < t_end; t += t_step) {
        if (__ldg(&P.recs[t].stop) <= step) continue;   // same skip rule as the producer
        bool ok = wait_full(sa, pa);   // the tile record is valid once its first unit has landed
        // every consumer warp is past the previous tile's E phase here; an abort anywhere ends the CTA
        if (bar_sync_or(2, NCT, !ok || *abort_flag != 0)) {
            if (threadIdx.x == 0) atomicOr(P.status, STATUS_TIMEOUT);
            return;
        }
        const TileRec *rec = &recs[m++ % NTR];
        const int x0 = rec->x0, y0 = rec->y0, kz0 = rec->kz0, kz1 = rec->kz1;
        const int nx = rec->nx, ny = rec->ny, nz = rec->nz;
        const long long pitch = rec->pitch, plane = rec->plane;
        const bool id_mode = rec->mode == COEF_ID8;
        const bool ch_uni = rec->ch_uniform != 0;
        if (id_mode && rec->table != tab_cached) {   // new cavity: copy its material table to shared memory
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
        const int gj = y0 + y;
        const int gi = x0 + x;
        const int kb = kz0 > 0 ? kz0 - 1 : kz0;

        auto at = [&](const T *base, int f, int xx, int yy) { return base + f * FE + yy * BX + xx; };
        auto ch_pair = [&](const uint8_t *ida_, int yy, float2 &cx, float2 &cy, float2 &cz) {
            cx = make_float2(ch_s0, ch_s0);
            cy = make_float2(ch_s1, ch_s1);
            cz = make_float2(ch_s2, ch_s2);
            if (id_mode && !ch_uni) {
                const uint32_t ip = *reinterpret_cast<const uint16_t *>(ida_ + (yy + 1) * G::IBX + x + G::IDX_HALO);
                const float4 a = table[2 * (ip & 0xff) + 1], b = table[2 * (ip >> 8) + 1];
                cx = make_float2(a.x, b.x);
                cy = make_float2(a.y, b.y);
                cz = make_float2(a.z, b.z);
            }
        };
        // halo row y = -1 of the plane held by units U (plane) and V (plane + 1): Hx and Hz only
        auto halo_row = [&](const T *U, const T *V, const uint8_t *idu, float *hbuf_) {
            const int ry = 0;   // box row of y = -1
            const float2 ey_ = Pair<T>::ld(at(U, 1, bx, ry)), ez_ = Pair<T>::ld(at(U, 2, bx, ry));
            const float2 ex_ = Pair<T>::ld(at(U, 0, bx, ry));
            const float2 ex_y1 = Pair<T>::ld(at(U, 0, bx, ry + 1)), ez_y1 = Pair<T>::ld(at(U, 2, bx, ry + 1));
            const float ey_x2 = Pair<T>::ld1(at(U, 1, bx + 2, ry));
            const float2 eyb = Pair<T>::ld(at(V, 1, bx, ry));
            float2 hx_ = Pair<T>::ld(at(U, 3, bx, ry)), hz_ = Pair<T>::ld(at(U, 5, bx, ry));
            float2 cx, cy, cz;
            ch_pair(idu, -1, cx, cy, cz);
            const float2 ey_x1 = make_float2(ey_.y, ey_x2);
            hx_ = fma2(cx, sub2(sub2(eyb, ey_), sub2(ez_y1, ez_)), hx_);
            hz_ = fma2(cz, sub2(sub2(ex_y1, ex_), sub2(ey_x1, ey_)), hz_);
            *reinterpret_cast<float2 *>(hbuf_ + x + 2) = hx_;
            *reinterpret_cast<float2 *>(hbuf_ + 2 * HC + x + 2) = hz_;
        };

        for (int k = kb; k < kz1; ++k) {
            int sb = sa + 1;
            uint32_t pb = pa;
            if (sb == S) {
                sb = 0;
                pb ^= 1u;
            }
            ok = wait_full(sa, pa) && wait_full(sb, pb);
            const bool prologue = k < kz0;
            const T *A = reinterpret_cast<const T *>(slots + sa * SB);
            const T *B = reinterpret_cast<const T *>(slots + sb * SB);
            const uint8_t *ida = slots + sa * SB + 6 * FS;
            float *hn = hbuf + hb * HB;
            float2 ex = make_float2(0.f, 0.f), ey = ex, ez = ex, hx = ex, hy = ex, hz = ex;
            uint32_t idpair = 0;

            // ---------------- phase A: H^{n+1/2} on own cells; the halo warp: row y = -1 and column x = -1
            if (!halo) {
                if (ok) {
                    ex = Pair<T>::ld(at(A, 0, bx, by));
                    ey = Pair<T>::ld(at(A, 1, bx, by));
                    ez = Pair<T>::ld(at(A, 2, bx, by));
                    const float2 ex_y1 = Pair<T>::ld(at(A, 0, bx, by + 1));
                    const float2 ez_y1 = Pair<T>::ld(at(A, 2, bx, by + 1));
                    const float ey_x2 = Pair<T>::ld1(at(A, 1, bx + 2, by));
                    const float ez_x2 = Pair<T>::ld1(at(A, 2, bx + 2, by));
                    const float2 exb = Pair<T>::ld(at(B, 0, bx, by));
                    const float2 eyb = Pair<T>::ld(at(B, 1, bx, by));
                    hx = Pair<T>::ld(at(A, 3, bx, by));
                    hy = Pair<T>::ld(at(A, 4, bx, by));
                    hz = Pair<T>::ld(at(A, 5, bx, by));
                    if (id_mode) idpair = *reinterpret_cast<const uint16_t *>(ida + by * G::IBX + x + G::IDX_HALO);
                    float2 chx, chy, chz;
                    ch_pair(ida, y, chx, chy, chz);
                    // packed over the lane's two cells; operand order makes each bracket -(curl E), so
                    // H + ch * bracket rounds exactly like H - ch * curl E
                    const float2 ez_x1 = make_float2(ez.y, ez_x2), ey_x1 = make_float2(ey.y, ey_x2);
                    hx = fma2(chx, sub2(sub2(eyb, ey), sub2(ez_y1, ez)), hx);
                    hy = fma2(chy, sub2(sub2(ez_x1, ez), sub2(exb, ex)), hy);
                    hz = fma2(chz, sub2(sub2(ex_y1, ex), sub2(ey_x1, ey)), hz);
                    const int o = by * HP + x + 2;
                    *reinterpret_cast<float2 *>(hn + o) = hx;
                    *reinterpret_cast<float2 *>(hn + HC + o) = hy;
                    *reinterpret_cast<float2 *>(hn + 2 * HC + o) = hz;
                    const long long g = (long long)k * plane + (long long)gj * pitch + gi;
                    if (!prologue && gj < ny && gi < nx && store_ok(P.status, g, 2, plane * nz)) {
                        Pair<T>::st(dst0 + g + 3 * fstride, hx.x, hx.y);
                        Pair<T>::st(dst0 + g + 4 * fstride, hy.x, hy.y);
                        Pair<T>::st(dst0 + g + 5 * fstride, hz.x, hz.y);
                    }
                }
            } else if (ok && !prologue) {
                halo_row(A, B, ida, hn);
                if (lane < TY) {
                    // column x = -1 of row yy: Hy and Hz (used by Ez and Ey at x = 0)
                    const int yy = lane, cbx = HX - 1, cby = yy + 1;
                    const float cex_ = Pair<T>::ld1(at(A, 0, cbx, cby));
                    const float cey_ = Pair<T>::ld1(at(A, 1, cbx, cby));
                    const float cez_ = Pair<T>::ld1(at(A, 2, cbx, cby));
                    const float cey_x1 = Pair<T>::ld1(at(A, 1, cbx + 1, cby));
                    const float cez_x1 = Pair<T>::ld1(at(A, 2, cbx + 1, cby));
                    const float cex_y1 = Pair<T>::ld1(at(A, 0, cbx, cby + 1));
                    const float cexb = Pair<T>::ld1(at(B, 0, cbx, cby));
                    float cchy = ch_s1, cchz = ch_s2;
                    if (id_mode && !ch_uni) {
                        const float4 a = table[2 * ida[cby * G::IBX + G::IDX_HALO - 1] + 1];
                        cchy = a.y;
                        cchz = a.z;
                    }
                    const float chy_ = Pair<T>::ld1(at(A, 4, cbx, cby)) -
                                       cchy * ((cexb - cex_) - (cez_x1 - cez_));
                    const float chz_ = Pair<T>::ld1(at(A, 5, cbx, cby)) -
                                       cchz * ((cey_x1 - cey_) - (cex_y1 - cex_));
                    hn[HC + cby * HP + 1] = chy_;
                    hn[2 * HC + cby * HP + 1] = chz_;
                }
            }
            // all of plane k's H (own rows, halo row and column) is in hn from here on
            asm volatile("bar.sync 1, %0;" ::"r"(NCT) : "memory");

            // ---------------- phase B: E^{n+1} on own cells (row warps)
            if (!halo) {
                if (ok && !prologue) {
                    const int o = by * HP + x + 2;
                    const float2 hx_ym = *reinterpret_cast<const float2 *>(hn + o - HP);
                    const float2 hz_ym = *reinterpret_cast<const float2 *>(hn + 2 * HC + o - HP);
                    const float hy_xm = hn[HC + o - 1];
                    const float hz_xm = hn[2 * HC + o - 1];
                    float4 ce_a = make_float4(ce_s0, ce_s1, ce_s2, 0.f), ce_b = ce_a;
                    if (id_mode) {
                        ce_a = table[2 * (idpair & 0xff)];
                        ce_b = table[2 * (idpair >> 8)];
                    }
                    // PEC: a zero coefficient leaves a tangential E exactly unchanged (e + 0 * c == e)
                    const bool k1 = k >= 1, j1 = gj >= 1, i1 = gi >= 1;
                    const float2 cex = (j1 && k1) ? make_float2(ce_a.x, ce_b.x) : make_float2(0.f, 0.f);
                    const float2 cey = make_float2((i1 && k1) ? ce_a.y : 0.f, k1 ? ce_b.y : 0.f);
                    const float2 cez = make_float2((i1 && j1) ? ce_a.z : 0.f, j1 ? ce_b.z : 0.f);
                    const float2 hz_xm2 = make_float2(hz_xm, hz.x), hy_xm2 = make_float2(hy_xm, hy.x);
                    ex = fma2(cex, sub2(sub2(hz, hz_ym), sub2(hy, hpy)), ex);
                    ey = fma2(cey, sub2(sub2(hx, hpx), sub2(hz, hz_xm2)), ey);
                    ez = fma2(cez, sub2(sub2(hy, hy_xm2), sub2(hx, hx_ym)), ez);
                    const long long g = (long long)k * plane + (long long)gj * pitch + gi;
                    if (gj < ny && gi < nx && store_ok(P.status, g, 2, plane * nz)) {
                        Pair<T>::st(dst0 + g, ex.x, ex.y);
                        Pair<T>::st(dst0 + g + 1 * fstride, ey.x, ey.y);
                        Pair<T>::st(dst0 + g + 2 * fstride, ez.x, ez.y);
                    }
                }
                hpx = hx;
                hpy = hy;
            }
            // ---------------- release the units this warp no longer reads
            const bool last = k == kz1 - 1;
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[sa]);
                if (last) mbar_arrive(&empty[sb]);
            }
            sa = sb;
            pa = pb;
            if (last && ++sa == S) {   // the tile's final unit (sb) is released too: move past it
                sa = 0;
                pa ^= 1u;
            }
            hb ^= 1;
        }
    }
}

template <typename T, int TY>
cudaError_t launch_typed(const FusedLaunch &L, cudaStream_t s) {
    const int smem = smem_bytes<T, TY>(L.stages);
    auto kern = fused_step_kernel<T, TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    FusedParams P;
    P.recs = L.recs;
    P.step = L.step;
    P.ntiles = L.ntiles;
    P.parity = L.parity;
    P.status = L.status;
    P.stages = L.stages;
    P.slot_bytes = slot_bytes<T, TY>();
    P.inject_timeout_us = L.inject_timeout_us;
    P.first = L.first;
    kern<<<L.grid, block_threads<TY>(), smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T, int TY>
cudaError_t occupancy_typed(int stages, int *n) {
    const int smem = smem_bytes<T, TY>(stages);
    auto kern = fused_step_kernel<T, TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, block_threads<TY>(), smem);
}

#define FDTD_DISPATCH(storage, tile_y, ...)                                                       \
    do {                                                                                          \
        if (storage == 0) {                                                                       \
            if (tile_y == 4) { using T = float; constexpr int TY = 4; __VA_ARGS__; }              \
            else if (tile_y == 8) { using T = float; constexpr int TY = 8; __VA_ARGS__; }         \
            else if (tile_y == 16) { using T = float; constexpr int TY = 16; __VA_ARGS__; }       \
        } else if (storage == 1) {                                                                \
            if (tile_y == 4) { using T = __half; constexpr int TY = 4; __VA_ARGS__; }             \
            else if (tile_y == 8) { using T = __half; constexpr int TY = 8; __VA_ARGS__; }        \
            else if (tile_y == 16) { using T = __half; constexpr int TY = 16; __VA_ARGS__; }      \
        } else if (storage == 2) {                                                                \
            if (tile_y == 4) { using T = __nv_bfloat16; constexpr int TY = 4; __VA_ARGS__; }      \
            else if (tile_y == 8) { using T = __nv_bfloat16; constexpr int TY = 8; __VA_ARGS__; } \
            else if (tile_y == 16) { using T = __nv_bfloat16; constexpr int TY = 16; __VA_ARGS__; } \
        }                                                                                         \
    } while (0)

}  // namespace

int fused_smem_bytes(int storage, int tile_y, int stages) {
    int r = -1;
    FDTD_DISPATCH(storage, tile_y, r = smem_bytes<T, TY>(stages));
    return r;
}

cudaError_t fused_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm) {
    cudaError_t e = cudaErrorInvalidValue;
    FDTD_DISPATCH(storage, tile_y, e = occupancy_typed<T, TY>(stages, ctas_per_sm));
    return e;
}

cudaError_t launch_fused_step(int storage, const FusedLaunch &L, cudaStream_t s) {
    if (L.ntiles <= 0) return cudaSuccess;
    if (L.stages < 3 || L.stages > 8) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    FDTD_DISPATCH(storage, L.tile_y, e = launch_typed<T, TY>(L, s));
    return e;
}

__global__ void step_counter_kernel(long long *c, int inc) { *c += inc; }

cudaError_t launch_step_counter(long long *counter, int inc, cudaStream_t s) {
    step_counter_kernel<<<1, 1, 0, s>>>(counter, inc);
    return cudaGetLastError();
}

void fused_box(int storage, int tile_y, int *box_x, int *box_y, int *halo_x) {
    const int esz = storage == 0 ? 4 : 2;
    *halo_x = 16 / esz;
    *box_x = TX + 2 * (16 / esz);
    *box_y = tile_y + 2;
}

}  // namespace fdtd
