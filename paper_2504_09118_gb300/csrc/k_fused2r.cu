// Two Yee leapfrog steps per pass over HBM, two rows per consumer warp, for sm_103a.
//
// The same computation as k_fused2.cu (Eq. 2 of the paper in the order of Listing 1, applied twice per
// launch: level 1 takes (H^{n-1/2}, E^n) to (H^{n+1/2}, E^{n+1}), level 2 takes that to (H^{n+3/2},
// E^{n+2}); PEC by index predicates; only level 2 is written, to copy 1-s), the same tiles, the same
// producer warp and TMA ring, the same operation sequence per value (so FP32 results are bit-identical
// to the one-row kernel and to two one-step launches).  What differs is the work split of the
// consumers: warp w owns the two adjacent rows r = 2w and 2w + 1 (y = y0 - 2 + r) instead of one.
//   * the per-plane skeleton (ring wait, two CTA barriers, slot arithmetic, phase predicates, the
//     release of the unit) is paid once per two rows;
//   * the y neighbour of the upper row is the lower row of the same warp: those H1, E1 and H2 values
//     pass in registers, and only the warp's edge rows go through shared planes (half the exchange
//     traffic, and shared memory left for a deeper TMA ring);
//   * the two rows are independent instruction streams, which hides latency with half the warps;
//   * the E coefficients of a level-1 E update (looked up by material id and masked at the PEC faces)
//     are kept in registers for the level-2 E update of the same plane one iteration later.
// Rows 0 .. TY + 2 are needed (TY even: the upper row of the last warp, TY + 3, is idle).
// It reads the two-step map set, so a context with PEC-coded material ids hands it those ids and their
// table (the tangential E coefficients on the faces already zero); its own masks then multiply the
// same zeros, and the results stay those of the one-row kernel.
//
// Per z-plane iteration k: [H1(k)] bar [E1(k)] [H2(k-1)] bar [E2(k-1) + stores], as in k_fused2.cu; the
// hazards on the shared planes are covered by the same two barriers (a plane written in one phase is
// read after the next barrier and rewritten only after the barrier that follows its last read).
#include "fused_common.cuh"
#include "launch.h"

namespace fdtd {

namespace {

using namespace fused;

constexpr int NTRR = 8;
constexpr uint64_t kWaitLimitNsR = 2000000000ull;

template <typename T> struct GeomR {
    static constexpr int HX = 16 / (int)sizeof(T);   // 4 (FP32) or 8 (16-bit): elements per 16-byte TMA granule
    static constexpr int W = 60;                      // output columns per tile
    // field box width: the lanes read box columns shift .. shift + 64 (the last one for the x + 1 neighbour),
    // and the origin shift is at most HX - 1, so 64 + HX columns cover every origin
    static constexpr int BX = 64 + HX;
    // The box starts at the lane cells' first column x0 - 2 rounded down to the 16-byte granule, so that every
    // tile origin (a multiple of 60) gives a legal TMA x coordinate; a lane's box column is shifted by the
    // remainder (2 for FP32, 0..6 for 16-bit storage).
    __host__ __device__ static constexpr int box_x(int x0) { return (x0 - 2) & ~(HX - 1); }
    static constexpr int IBX = 80;                    // id box width (bytes)
};

struct FusedRParams {
    const TileRec *recs;
    const long long *step;   // batch step clock (NULL: a single cavity, no tile is skipped)
    int launch_steps;        // 2, or 1: level 1 only
    int ntiles;
    int parity;
    int *status;
    int stages;
    int slot_bytes;
    const int *first;   // per-CTA tile ranges (NULL: round-robin)
};

__host__ __device__ constexpr int alr(int v, int a) { return (v + a - 1) / a * a; }

template <typename T, int TY> __host__ __device__ constexpr int boxr_bytes() {
    return GeomR<T>::BX * (TY + 4) * (int)sizeof(T);
}
template <int TY> __host__ __device__ constexpr int idboxr_bytes() { return GeomR<float>::IBX * (TY + 4); }
// six field boxes back to back (one 4-D load), then the id box at the next 128-byte boundary
template <typename T, int TY> __host__ __device__ constexpr int idboxr_off() { return alr(6 * boxr_bytes<T, TY>(), 128); }
template <typename T, int TY> __host__ __device__ constexpr int slotr_bytes() {
    return alr(idboxr_off<T, TY>() + idboxr_bytes<TY>(), 128);
}
template <int TY> __host__ __device__ constexpr int nwarps_r() { return (TY + 4) / 2; }   // consumer warps
constexpr int PWR = 68;   // shared plane row pitch: column x - x0 + 4 (lane cells at 2 lane + 2, + 3)
// exchange planes, one row per warp boundary (NW + 1 rows): H1 (Hx, Hz), H2 (Hx, Hz), E1 (Ex, Ez) x 2
template <int TY> __host__ __device__ constexpr int planer_floats() { return (nwarps_r<TY>() + 1) * PWR; }
constexpr int TABR_BYTES = kMaxTable * 2 * 16;
template <typename T, int TY> __host__ __device__ constexpr int smemr_bytes(int stages) {
    // barriers/abort | records | table | exchange planes | ring
    return 256 + NTRR * (int)sizeof(TileRec) + TABR_BYTES + alr(8 * planer_floats<TY>() * 4, 128) +
           stages * slotr_bytes<T, TY>();
}
template <int TY> __host__ __device__ constexpr int threadsr() { return (nwarps_r<TY>() + 1) * 32; }

// Values of one row that live across z-planes.
struct RowCarry {
    float2 h1x, h1y, h1z;     // H1(k-1)
    float2 e1x, e1y, e1z;     // E1(k-1)
    float2 h2x, h2y;          // H2(k-2) (Hx, Hy)
    float2 cex, cey, cez;     // masked ce of E1(k-1), reused by E2(k-1)
    uint32_t id;              // material ids of plane k-1
};

template <typename T, int TY, bool BATCH>
__global__ void __launch_bounds__(threadsr<TY>(), 1) fused2r_step_kernel(const FusedRParams P) {
    using G = GeomR<T>;
    constexpr int BX = G::BX, W = G::W;
    constexpr int FB = boxr_bytes<T, TY>(), FE = FB / (int)sizeof(T), IDO = idboxr_off<T, TY>();
    static_assert(FB % 16 == 0 && FE % 2 == 0, "field boxes keep 16-byte rows and even-aligned pairs");
    constexpr int NW = nwarps_r<TY>(), NCT = NW * 32;
    constexpr int PF = planer_floats<TY>();
    static_assert(2 * NW == TY + 4, "rows 0 .. TY + 3 in pairs");

    extern __shared__ __align__(128) unsigned char smem[];
    if (smem_u32(smem) & 127u) {
        if (threadIdx.x == 0) atomicOr(P.status, STATUS_BADINDEX);
        return;
    }
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 8;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 128);
    TileRec *recs = reinterpret_cast<TileRec *>(smem + 256);
    float4 *stab = reinterpret_cast<float4 *>(smem + 256 + NTRR * sizeof(TileRec));
    float *planes = reinterpret_cast<float *>(smem + 256 + NTRR * sizeof(TileRec) + TABR_BYTES);
    float *sh1x = planes, *sh1z = planes + PF, *sh2x = planes + 2 * PF, *sh2z = planes + 3 * PF;
    float *e1b = planes + 4 * PF;   // [buffer][Ex, Ez][PF]
    unsigned char *slots = smem + 256 + NTRR * sizeof(TileRec) + TABR_BYTES + alr(8 * PF * 4, 128);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = P.stages, SB = P.slot_bytes;
    const int t_begin = P.first ? __ldg(P.first + blockIdx.x) : (int)blockIdx.x;
    const int t_end = P.first ? __ldg(P.first + blockIdx.x + 1) : P.ntiles;
    const int t_step = P.first ? 1 : (int)gridDim.x;
    const long long clock = BATCH ? *P.step : 0;

    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        fence_mbarrier_init();
        fence_proxy_async_smem();
    }
    __syncthreads();

    // =========================================================== producer warp (as in k_fused2.cu)
    if (warp == NW) {
        int issued = 0, m = 0, s = 0;
        uint32_t rnd = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; t += t_step) {
            if (BATCH && __ldg(&P.recs[t].stop) <= clock) continue;
            TileRec *rec = &recs[m++ % NTRR];
            int kb = 0, klast = 0;
            for (int k = 0;; ++k) {
                if (issued >= S) {
                    const bool w = mbar_wait_abortable(&empty[s], rnd ^ 1u, kWaitLimitNsR, abort_flag, 0);
                    if (!__all_sync(0xffffffffu, w)) {
                        ok = false;
                        break;
                    }
                }
                if (__any_sync(0xffffffffu, *abort_flag != 0)) {
                    ok = false;
                    break;
                }
                if (k == 0) {
                    const uint32_t *src = reinterpret_cast<const uint32_t *>(P.recs + t);
                    uint32_t *dst = reinterpret_cast<uint32_t *>(rec);
                    for (int q = lane; q < (int)(sizeof(TileRec) / 4); q += 32) dst[q] = __ldg(src + q);
                    __syncwarp();
                    kb = rec->kz0 > 2 ? rec->kz0 - 2 : 0;
                    klast = rec->kz1 + 1;
                }
                const int kk = kb + k;
                if (lane == 0) {
                    const int src_copy = P.parity ^ rec->parity_off;
                    const bool has_id = rec->mode == COEF_ID8;
                    unsigned char *dst = slots + s * SB;
                    fence_proxy_async_smem();
                    if (tma_x_ok(P.status, G::box_x(rec->x0), (int)sizeof(T)) &&
                        (!has_id || tma_x_ok(P.status, rec->id_x0, 1))) {
                        mbar_arrive_expect_tx(&full[s], 6 * FB + (has_id ? idboxr_bytes<TY>() : 0));
                        tma_load_4d(dst, rec->maps + src_copy * 6, G::box_x(rec->x0), rec->y0 - 2, kk, 0, &full[s]);
                        if (has_id)
                            tma_load_3d(dst + IDO, rec->maps + 12, rec->id_x0, rec->y0 - 2, kk, &full[s]);
                    } else {
                        mbar_arrive(&full[s]);
                    }
                }
                __syncwarp();
                ++issued;
                if (++s == S) {
                    s = 0;
                    rnd ^= 1u;
                }
                if (kk >= klast) break;
            }
        }
        if (!ok && lane == 0) {
            atomicOr(P.status, STATUS_TIMEOUT);
            for (int u = issued > S ? issued - S : 0; u < issued; ++u)
                mbar_wait_bounded(&full[u % S], (u / S) & 1, kWaitLimitNsR);
        }
        return;
    }

    // =========================================================== consumer warps: rows ra = 2w, rb = 2w + 1
    const int ra = 2 * warp, rb = ra + 1;
    const bool b_live = rb <= TY + 2;        // warp-uniform; false only for the last warp's upper row
    const int pc = 2 * lane + 2;             // shared plane column of the first cell
    float *const sh1x_w = sh1x + (warp + 1) * PWR + pc, *const sh1z_w = sh1z + (warp + 1) * PWR + pc;
    const float *const sh1x_r = sh1x + warp * PWR + pc, *const sh1z_r = sh1z + warp * PWR + pc;
    float *const sh2x_w = sh2x + (warp + 1) * PWR + pc, *const sh2z_w = sh2z + (warp + 1) * PWR + pc;
    const float *const sh2x_r = sh2x + warp * PWR + pc, *const sh2z_r = sh2z + warp * PWR + pc;
    int sa = 0, m = 0;
    uint32_t pa = 0;
    const float4 *tab_cached = nullptr;
    auto wait_full = [&](int slot, uint32_t par) {
        return mbar_wait_abortable(&full[slot], par, kWaitLimitNsR, abort_flag, 0);
    };
    const float2 zero2 = make_float2(0.f, 0.f);

    for (int t = t_begin; t < t_end; t += t_step) {
        if (BATCH && __ldg(&P.recs[t].stop) <= clock) continue;
        bool ok = wait_full(sa, pa);
        if (bar_sync_or(2, NCT, !ok || *abort_flag != 0)) {
            if (threadIdx.x == 0) atomicOr(P.status, STATUS_TIMEOUT);
            return;
        }
        const TileRec *rec = &recs[m++ % NTRR];
        const int x0 = rec->x0, y0 = rec->y0, kz0 = rec->kz0, kz1 = rec->kz1;
        const int bx = (x0 - 2) - G::box_x(x0) + 2 * lane;   // box column of the lane's first cell
        const int nx = rec->nx, ny = rec->ny, nz = rec->nz;
        const long long pitch = rec->pitch, plane = rec->plane;
        const bool id_mode = rec->mode == COEF_ID8;
        const bool ch_uni = rec->ch_uniform != 0;
        const int idoff = x0 - 2 - rec->id_x0;
        if (id_mode && rec->table != tab_cached) {
            const float4 *src = rec->table;
            const int n = 2 * rec->ntab;
            for (int e = threadIdx.x; e < n; e += NCT) stab[e] = __ldg(src + e);
            bar_sync_or(2, NCT, false);
            tab_cached = src;
        }
        const int dstc = (P.parity ^ rec->parity_off) ^ 1;
        T *const dst0 = static_cast<T *>(rec->dst[dstc][0]);
        const long long fstride = plane * nz;
        const float4 ce_s = make_float4(rec->ce[0], rec->ce[1], rec->ce[2], 0.f);
        const float4 ch_s = make_float4(rec->ch[0], rec->ch[1], rec->ch[2], 0.f);
        const int gja = y0 - 2 + ra, gjb = gja + 1;
        const int gi = x0 - 2 + 2 * lane;
        const bool ina = gi >= 0 && gi < nx, inb = gi + 1 < nx;
        const bool i1a = gi >= 1;
        const bool out_a = lane >= 1 && 2 * lane - 2 < W && gi < nx;
        // per row: stored level-2 row, E1 row (r >= 1), H2 row (1 <= r <= TY + 1)
        const bool outr_a = ra >= 2 && ra < TY + 2 && gja < ny, outr_b = rb >= 2 && rb < TY + 2 && gjb < ny;
        const bool e1r_a = ra >= 1, e1r_b = b_live;
        const bool h2r_a = ra >= 1 && ra <= TY + 1, h2r_b = rb <= TY + 1;
        const bool rowin_a = gja >= 0 && gja < ny, rowin_b = gjb >= 0 && gjb < ny;
        const bool j1a = gja >= 1, j1b = gjb >= 1;
        const int kb = kz0 > 2 ? kz0 - 2 : 0;
        const bool level1_only = BATCH && (P.launch_steps == 1 || rec->stop - clock == 1);

        auto at = [&](const T *base, int f, int xx, int yy) { return base + f * FE + yy * BX + xx; };
        auto coef = [&](uint32_t ip, int which, float4 &a, float4 &b) {   // which: 0 ce, 1 ch
            if (id_mode && !(which && ch_uni)) {
                a = stab[2 * (ip & 0xff) + which];
                b = stab[2 * (ip >> 8) + which];
            } else {
                a = b = which ? ch_s : ce_s;
            }
        };
        RowCarry A_{}, B_{};   // rows a and b

#pragma unroll 1
        for (int k = kb; k <= kz1; ++k) {
            int sb = sa + 1;
            uint32_t pb = pa;
            if (sb == S) {
                sb = 0;
                pb ^= 1u;
            }
            ok = wait_full(sb, pb);
            ok = __all_sync(0xffffffffu, ok);
            const T *Au = reinterpret_cast<const T *>(slots + sa * SB);
            const T *Bu = reinterpret_cast<const T *>(slots + sb * SB);
            const uint8_t *ida = slots + sa * SB + IDO;
            const bool do_e1 = k >= kz0 - 1;
            const bool do_h2 = !level1_only && k >= kz0 && k >= 1, do_e2 = !level1_only && k >= kz0 + 1;
            float *e1cur = e1b + (k & 1) * 2 * PF, *e1prv = e1b + ((k + 1) & 1) * 2 * PF;
            const bool k1 = k >= 1, inz = k < nz;

            // ---------------- phase 1: H1(k) on rows a and b
            float2 ex_a = zero2, ey_a = zero2, ez_a = zero2, hx_a = zero2, hy_a = zero2, hz_a = zero2;
            float2 ex_b = zero2, ey_b = zero2, ez_b = zero2, hx_b = zero2, hy_b = zero2, hz_b = zero2;
            uint32_t id_a = 0, id_b = 0;
            if (ok) {
                ex_a = Pair<T>::ld(at(Au, 0, bx, ra));
                ey_a = Pair<T>::ld(at(Au, 1, bx, ra));
                ez_a = Pair<T>::ld(at(Au, 2, bx, ra));
                ex_b = Pair<T>::ld(at(Au, 0, bx, rb));
                ey_b = Pair<T>::ld(at(Au, 1, bx, rb));
                ez_b = Pair<T>::ld(at(Au, 2, bx, rb));
                hx_a = Pair<T>::ld(at(Au, 3, bx, ra));
                hy_a = Pair<T>::ld(at(Au, 4, bx, ra));
                hz_a = Pair<T>::ld(at(Au, 5, bx, ra));
                const float ey_x2a = Pair<T>::ld1(at(Au, 1, bx + 2, ra));
                const float ez_x2a = Pair<T>::ld1(at(Au, 2, bx + 2, ra));
                const float2 exz_a = Pair<T>::ld(at(Bu, 0, bx, ra));
                const float2 eyz_a = Pair<T>::ld(at(Bu, 1, bx, ra));
                if (id_mode) {
                    id_a = *reinterpret_cast<const uint16_t *>(ida + ra * G::IBX + idoff + 2 * lane);
                    id_b = *reinterpret_cast<const uint16_t *>(ida + rb * G::IBX + idoff + 2 * lane);
                }
                float4 ca, cb;
                coef(id_a, 1, ca, cb);
                const float2 ez_x1 = make_float2(ez_a.y, ez_x2a), ey_x1 = make_float2(ey_a.y, ey_x2a);
                // row a's y + 1 neighbours are row b's own values
                hx_a = fma2(make_float2(ca.x, cb.x), sub2(sub2(eyz_a, ey_a), sub2(ez_b, ez_a)), hx_a);
                hy_a = fma2(make_float2(ca.y, cb.y), sub2(sub2(ez_x1, ez_a), sub2(exz_a, ex_a)), hy_a);
                hz_a = fma2(make_float2(ca.z, cb.z), sub2(sub2(ex_b, ex_a), sub2(ey_x1, ey_a)), hz_a);
                if (b_live) {
                    hx_b = Pair<T>::ld(at(Au, 3, bx, rb));
                    hy_b = Pair<T>::ld(at(Au, 4, bx, rb));
                    hz_b = Pair<T>::ld(at(Au, 5, bx, rb));
                    const float2 ex_y1 = Pair<T>::ld(at(Au, 0, bx, rb + 1));
                    const float2 ez_y1 = Pair<T>::ld(at(Au, 2, bx, rb + 1));
                    const float ey_x2b = Pair<T>::ld1(at(Au, 1, bx + 2, rb));
                    const float ez_x2b = Pair<T>::ld1(at(Au, 2, bx + 2, rb));
                    const float2 exz_b = Pair<T>::ld(at(Bu, 0, bx, rb));
                    const float2 eyz_b = Pair<T>::ld(at(Bu, 1, bx, rb));
                    coef(id_b, 1, ca, cb);
                    const float2 ez_x1b = make_float2(ez_b.y, ez_x2b), ey_x1b = make_float2(ey_b.y, ey_x2b);
                    hx_b = fma2(make_float2(ca.x, cb.x), sub2(sub2(eyz_b, ey_b), sub2(ez_y1, ez_b)), hx_b);
                    hy_b = fma2(make_float2(ca.y, cb.y), sub2(sub2(ez_x1b, ez_b), sub2(exz_b, ex_b)), hy_b);
                    hz_b = fma2(make_float2(ca.z, cb.z), sub2(sub2(ex_y1, ex_b), sub2(ey_x1b, ey_b)), hz_b);
                    *reinterpret_cast<float2 *>(sh1x_w) = hx_b;
                    *reinterpret_cast<float2 *>(sh1z_w) = hz_b;
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(NCT) : "memory");

            // ---------------- phase 2: E1(k) (zero outside the cavity: tangential at its far faces)
            float2 e1x_a = zero2, e1y_a = zero2, e1z_a = zero2, e1x_b = zero2, e1y_b = zero2, e1z_b = zero2;
            float2 cex_a = zero2, cey_a = zero2, cez_a = zero2, cex_b = zero2, cey_b = zero2, cez_b = zero2;
            if (ok && do_e1) {
                const float hz_xma = __shfl_up_sync(0xffffffffu, hz_a.y, 1);
                const float hy_xma = __shfl_up_sync(0xffffffffu, hy_a.y, 1);
                const float hz_xmb = __shfl_up_sync(0xffffffffu, hz_b.y, 1);
                const float hy_xmb = __shfl_up_sync(0xffffffffu, hy_b.y, 1);
                float4 ca, cb;
                if (e1r_a) {
                    const float2 hx_ym = *reinterpret_cast<const float2 *>(sh1x_r);
                    const float2 hz_ym = *reinterpret_cast<const float2 *>(sh1z_r);
                    coef(id_a, 0, ca, cb);
                    cex_a = make_float2((j1a && k1) ? ca.x : 0.f, (j1a && k1) ? cb.x : 0.f);
                    cey_a = make_float2((i1a && k1) ? ca.y : 0.f, k1 ? cb.y : 0.f);
                    cez_a = make_float2((i1a && j1a) ? ca.z : 0.f, j1a ? cb.z : 0.f);
                    e1x_a = fma2(cex_a, sub2(sub2(hz_a, hz_ym), sub2(hy_a, A_.h1y)), ex_a);
                    e1y_a = fma2(cey_a, sub2(sub2(hx_a, A_.h1x), sub2(hz_a, make_float2(hz_xma, hz_a.x))), ey_a);
                    e1z_a = fma2(cez_a, sub2(sub2(hy_a, make_float2(hy_xma, hy_a.x)), sub2(hx_a, hx_ym)), ez_a);
                    const bool va = rowin_a && ina && inz, vb = rowin_a && inb && inz;
                    if (!va) { e1x_a.x = 0.f; e1y_a.x = 0.f; e1z_a.x = 0.f; }
                    if (!vb) { e1x_a.y = 0.f; e1y_a.y = 0.f; e1z_a.y = 0.f; }
                    *reinterpret_cast<float2 *>(e1cur + warp * PWR + pc) = e1x_a;
                    *reinterpret_cast<float2 *>(e1cur + PF + warp * PWR + pc) = e1z_a;
                }
                if (e1r_b) {
                    coef(id_b, 0, ca, cb);
                    cex_b = make_float2((j1b && k1) ? ca.x : 0.f, (j1b && k1) ? cb.x : 0.f);
                    cey_b = make_float2((i1a && k1) ? ca.y : 0.f, k1 ? cb.y : 0.f);
                    cez_b = make_float2((i1a && j1b) ? ca.z : 0.f, j1b ? cb.z : 0.f);
                    // row b's y - 1 neighbours are row a's H1
                    e1x_b = fma2(cex_b, sub2(sub2(hz_b, hz_a), sub2(hy_b, B_.h1y)), ex_b);
                    e1y_b = fma2(cey_b, sub2(sub2(hx_b, B_.h1x), sub2(hz_b, make_float2(hz_xmb, hz_b.x))), ey_b);
                    e1z_b = fma2(cez_b, sub2(sub2(hy_b, make_float2(hy_xmb, hy_b.x)), sub2(hx_b, hx_a)), ez_b);
                    const bool va = rowin_b && ina && inz, vb = rowin_b && inb && inz;
                    if (!va) { e1x_b.x = 0.f; e1y_b.x = 0.f; e1z_b.x = 0.f; }
                    if (!vb) { e1x_b.y = 0.f; e1y_b.y = 0.f; e1z_b.y = 0.f; }
                }
                if (level1_only && out_a && k >= kz0 && k < kz1) {   // one step: (H1, E1) is the result
                    const long long g = (long long)k * plane + (long long)gja * pitch + gi;
                    if (outr_a && store_ok(P.status, g, 2, plane * nz)) {
                        Pair<T>::st_cs(dst0 + g, e1x_a.x, e1x_a.y);
                        Pair<T>::st_cs(dst0 + g + 1 * fstride, e1y_a.x, e1y_a.y);
                        Pair<T>::st_cs(dst0 + g + 2 * fstride, e1z_a.x, e1z_a.y);
                        Pair<T>::st_cs(dst0 + g + 3 * fstride, hx_a.x, hx_a.y);
                        Pair<T>::st_cs(dst0 + g + 4 * fstride, hy_a.x, hy_a.y);
                        Pair<T>::st_cs(dst0 + g + 5 * fstride, hz_a.x, hz_a.y);
                    }
                    const long long gb = g + pitch;
                    if (outr_b && store_ok(P.status, gb, 2, plane * nz)) {
                        Pair<T>::st_cs(dst0 + gb, e1x_b.x, e1x_b.y);
                        Pair<T>::st_cs(dst0 + gb + 1 * fstride, e1y_b.x, e1y_b.y);
                        Pair<T>::st_cs(dst0 + gb + 2 * fstride, e1z_b.x, e1z_b.y);
                        Pair<T>::st_cs(dst0 + gb + 3 * fstride, hx_b.x, hx_b.y);
                        Pair<T>::st_cs(dst0 + gb + 4 * fstride, hy_b.x, hy_b.y);
                        Pair<T>::st_cs(dst0 + gb + 5 * fstride, hz_b.x, hz_b.y);
                    }
                }
            }
            // No barrier here (as in k_fused2.cu): phase 3 reads this warp's own E1 values and the
            // row above's E1(k-1), written in the previous iteration into the other E1 buffer.

            // ---------------- phase 3: H2(k-1) = H1(k-1) - ch curl E1 (plane k-1, z+1 from plane k)
            float2 h2x_a = zero2, h2y_a = zero2, h2z_a = zero2, h2x_b = zero2, h2y_b = zero2, h2z_b = zero2;
            if (ok && do_h2) {
                const float ey_x2a = __shfl_down_sync(0xffffffffu, A_.e1y.x, 1);
                const float ez_x2a = __shfl_down_sync(0xffffffffu, A_.e1z.x, 1);
                const float ey_x2b = __shfl_down_sync(0xffffffffu, B_.e1y.x, 1);
                const float ez_x2b = __shfl_down_sync(0xffffffffu, B_.e1z.x, 1);
                float4 ca, cb;
                if (h2r_a) {
                    coef(A_.id, 1, ca, cb);
                    const float2 ez_x1 = make_float2(A_.e1z.y, ez_x2a), ey_x1 = make_float2(A_.e1y.y, ey_x2a);
                    // row a's y + 1 neighbour at plane k - 1 is row b's E1(k-1)
                    h2x_a = fma2(make_float2(ca.x, cb.x), sub2(sub2(e1y_a, A_.e1y), sub2(B_.e1z, A_.e1z)), A_.h1x);
                    h2y_a = fma2(make_float2(ca.y, cb.y), sub2(sub2(ez_x1, A_.e1z), sub2(e1x_a, A_.e1x)), A_.h1y);
                    h2z_a = fma2(make_float2(ca.z, cb.z), sub2(sub2(B_.e1x, A_.e1x), sub2(ey_x1, A_.e1y)), A_.h1z);
                }
                if (h2r_b) {
                    const float2 ex_y1 = *reinterpret_cast<const float2 *>(e1prv + (warp + 1) * PWR + pc);
                    const float2 ez_y1 = *reinterpret_cast<const float2 *>(e1prv + PF + (warp + 1) * PWR + pc);
                    coef(B_.id, 1, ca, cb);
                    const float2 ez_x1 = make_float2(B_.e1z.y, ez_x2b), ey_x1 = make_float2(B_.e1y.y, ey_x2b);
                    h2x_b = fma2(make_float2(ca.x, cb.x), sub2(sub2(e1y_b, B_.e1y), sub2(ez_y1, B_.e1z)), B_.h1x);
                    h2y_b = fma2(make_float2(ca.y, cb.y), sub2(sub2(ez_x1, B_.e1z), sub2(e1x_b, B_.e1x)), B_.h1y);
                    h2z_b = fma2(make_float2(ca.z, cb.z), sub2(sub2(ex_y1, B_.e1x), sub2(ey_x1, B_.e1y)), B_.h1z);
                    *reinterpret_cast<float2 *>(sh2x_w) = h2x_b;
                    *reinterpret_cast<float2 *>(sh2z_w) = h2z_b;
                }
            }
            const float h2z_xma = __shfl_up_sync(0xffffffffu, h2z_a.y, 1);
            const float h2y_xma = __shfl_up_sync(0xffffffffu, h2y_a.y, 1);
            const float h2z_xmb = __shfl_up_sync(0xffffffffu, h2z_b.y, 1);
            const float h2y_xmb = __shfl_up_sync(0xffffffffu, h2y_b.y, 1);
            asm volatile("bar.sync 1, %0;" ::"r"(NCT) : "memory");

            // ---------------- phase 4: E2(k-1) = E1(k-1) + ce curl H2, and the level-2 stores
            if (ok && do_e2 && out_a) {
                const long long g = (long long)(k - 1) * plane + (long long)gja * pitch + gi;
                if (outr_a) {
                    const float2 hx_ym = *reinterpret_cast<const float2 *>(sh2x_r);
                    const float2 hz_ym = *reinterpret_cast<const float2 *>(sh2z_r);
                    const float2 e2x = fma2(A_.cex, sub2(sub2(h2z_a, hz_ym), sub2(h2y_a, A_.h2y)), A_.e1x);
                    const float2 e2y =
                        fma2(A_.cey, sub2(sub2(h2x_a, A_.h2x), sub2(h2z_a, make_float2(h2z_xma, h2z_a.x))), A_.e1y);
                    const float2 e2z =
                        fma2(A_.cez, sub2(sub2(h2y_a, make_float2(h2y_xma, h2y_a.x)), sub2(h2x_a, hx_ym)), A_.e1z);
                    if (store_ok(P.status, g, 2, plane * nz)) {
                        Pair<T>::st_cs(dst0 + g, e2x.x, e2x.y);
                        Pair<T>::st_cs(dst0 + g + 1 * fstride, e2y.x, e2y.y);
                        Pair<T>::st_cs(dst0 + g + 2 * fstride, e2z.x, e2z.y);
                        Pair<T>::st_cs(dst0 + g + 3 * fstride, h2x_a.x, h2x_a.y);
                        Pair<T>::st_cs(dst0 + g + 4 * fstride, h2y_a.x, h2y_a.y);
                        Pair<T>::st_cs(dst0 + g + 5 * fstride, h2z_a.x, h2z_a.y);
                    }
                }
                if (outr_b) {
                    // row b's y - 1 neighbours are row a's H2
                    const float2 e2x = fma2(B_.cex, sub2(sub2(h2z_b, h2z_a), sub2(h2y_b, B_.h2y)), B_.e1x);
                    const float2 e2y =
                        fma2(B_.cey, sub2(sub2(h2x_b, B_.h2x), sub2(h2z_b, make_float2(h2z_xmb, h2z_b.x))), B_.e1y);
                    const float2 e2z =
                        fma2(B_.cez, sub2(sub2(h2y_b, make_float2(h2y_xmb, h2y_b.x)), sub2(h2x_b, h2x_a)), B_.e1z);
                    const long long gb = g + pitch;
                    if (store_ok(P.status, gb, 2, plane * nz)) {
                        Pair<T>::st_cs(dst0 + gb, e2x.x, e2x.y);
                        Pair<T>::st_cs(dst0 + gb + 1 * fstride, e2y.x, e2y.y);
                        Pair<T>::st_cs(dst0 + gb + 2 * fstride, e2z.x, e2z.y);
                        Pair<T>::st_cs(dst0 + gb + 3 * fstride, h2x_b.x, h2x_b.y);
                        Pair<T>::st_cs(dst0 + gb + 4 * fstride, h2y_b.x, h2y_b.y);
                        Pair<T>::st_cs(dst0 + gb + 5 * fstride, h2z_b.x, h2z_b.y);
                    }
                }
            }
            // ---------------- carry the z neighbours to the next plane
            A_.h2x = h2x_a; A_.h2y = h2y_a;
            A_.h1x = hx_a; A_.h1y = hy_a; A_.h1z = hz_a;
            A_.e1x = e1x_a; A_.e1y = e1y_a; A_.e1z = e1z_a;
            A_.cex = cex_a; A_.cey = cey_a; A_.cez = cez_a;
            A_.id = id_a;
            B_.h2x = h2x_b; B_.h2y = h2y_b;
            B_.h1x = hx_b; B_.h1y = hy_b; B_.h1z = hz_b;
            B_.e1x = e1x_b; B_.e1y = e1y_b; B_.e1z = e1z_b;
            B_.cex = cex_b; B_.cey = cey_b; B_.cez = cez_b;
            B_.id = id_b;
            // ---------------- release unit k (and k+1 after the last plane)
            const bool last = k == kz1;
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[sa]);
                if (last) mbar_arrive(&empty[sb]);
            }
            sa = sb;
            pa = pb;
            if (last && ++sa == S) {
                sa = 0;
                pa ^= 1u;
            }
        }
    }
}

template <typename T, int TY, bool BATCH>
cudaError_t launchr_typed(const FusedLaunch &L, cudaStream_t s) {
    const int smem = smemr_bytes<T, TY>(L.stages);
    auto kern = fused2r_step_kernel<T, TY, BATCH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    FusedRParams P;
    P.recs = L.recs;
    P.step = L.step;
    P.launch_steps = L.launch_steps == 1 ? 1 : 2;
    P.ntiles = L.ntiles;
    P.parity = L.parity;
    P.status = L.status;
    P.stages = L.stages;
    P.slot_bytes = slotr_bytes<T, TY>();
    P.first = L.first;
    kern<<<L.grid, threadsr<TY>(), smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T, int TY>
cudaError_t occupancyr_typed(int stages, int *n) {
    const int smem = smemr_bytes<T, TY>(stages);
    auto kern = fused2r_step_kernel<T, TY, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, threadsr<TY>(), smem);
}

#define FDTD_DISPATCHR(storage, tile_y, ...)                                                          \
    do {                                                                                              \
        if (storage == 0) {                                                                           \
            if (tile_y == 12) { using T = float; constexpr int TY = 12; __VA_ARGS__; }                \
            else if (tile_y == 16) { using T = float; constexpr int TY = 16; __VA_ARGS__; }           \
        } else if (storage == 1) {                                                                    \
            if (tile_y == 12) { using T = __half; constexpr int TY = 12; __VA_ARGS__; }               \
            else if (tile_y == 16) { using T = __half; constexpr int TY = 16; __VA_ARGS__; }          \
        } else if (storage == 2) {                                                                    \
            if (tile_y == 12) { using T = __nv_bfloat16; constexpr int TY = 12; __VA_ARGS__; }        \
            else if (tile_y == 16) { using T = __nv_bfloat16; constexpr int TY = 16; __VA_ARGS__; }   \
        }                                                                                             \
    } while (0)

}  // namespace

int fused2r_smem_bytes(int storage, int tile_y, int stages) {
    int r = -1;
    FDTD_DISPATCHR(storage, tile_y, r = smemr_bytes<T, TY>(stages));
    return r;
}

cudaError_t fused2r_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm) {
    cudaError_t e = cudaErrorInvalidValue;
    FDTD_DISPATCHR(storage, tile_y, e = occupancyr_typed<T, TY>(stages, ctas_per_sm));
    return e;
}

cudaError_t launch_fused2r_step(int storage, const FusedLaunch &L, cudaStream_t s) {
    if (L.ntiles <= 0) return cudaSuccess;
    if (L.stages < 3 || L.stages > 8) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    if (L.step || L.launch_steps == 1)
        FDTD_DISPATCHR(storage, L.tile_y, e = (launchr_typed<T, TY, true>(L, s)));
    else
        FDTD_DISPATCHR(storage, L.tile_y, e = (launchr_typed<T, TY, false>(L, s)));
    return e;
}

}  // namespace fdtd
