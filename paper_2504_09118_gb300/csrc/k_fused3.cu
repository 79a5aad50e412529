// Three Yee leapfrog steps per pass over HBM (temporal blocking, T = 3) for sm_103a, single cavities.
// Tile heights 8, 10 (16 warps: the 128-register cap) and 12 (18 warps: 96 registers, a small spill).
//
// The update of Eq. 2 in the order of Listing 1 (PEC by index predicates), applied three times per
// launch: level l takes (H^{n+l-3/2}, E^{n+l-1}) to (H^{n+l-1/2}, E^{n+l}); only level 3 is written to HBM
// (copy 1-s), so a step moves a third of the one-step kernel's DRAM bytes, at the price of a halo three
// cells wide at level 1.  Every value goes through the same operations in the same order as in the one-
// and two-step kernels, so FP32 results are bit-identical to theirs.
//
// Tile: W = 58 output columns x TY output rows over planes [kz0, kz1).  Each lane owns the two cells
// x0 - 4 + 2 lane, +1 (an even start keeps the 16-bit pairs aligned); the TMA box starts at x0 - 4
// rounded down to the 16-byte granule and is 64 + one granule wide.  Consumer warps r = 0..TY+4 own rows
// y = y0 - 3 + r.  Each level loses one valid cell per half step on the side its difference reaches:
//   H1 rows 0..TY+4   E1 rows 1..TY+4   H2 rows 1..TY+3   E2 rows 2..TY+3   H3 rows 2..TY+2   E3 rows 3..TY+2
// (and likewise in x), so rows 3..TY+2 and columns x0 .. x0 + 57 are exact.  E1 and E2 outside the cavity
// are forced to 0 (tangential at the far faces, nothing beyond them).
//
// Per z-plane iteration k:
//   [H1(k)] bar [E1(k), H2(k-1)] bar [E2(k-1), H3(k-2)] bar [E3(k-2) + stores]
// H2(k-1) reads the row below's E1(k-1) (written the iteration before, double-buffered) and H3(k-2) the
// row below's E2(k-2) (likewise), so the three barriers cover every shared-plane dependency.  A producer
// warp streams plane units (six field boxes with a 3-cell halo in y, one 4-D TMA load, and the id box)
// through an S-slot ring; waits are bounded and a shared abort flag ends the CTA together.
#include "fused_common.cuh"
#include "launch.h"

namespace fdtd {

namespace {

using namespace fused;

constexpr int NTR3 = 8;
constexpr uint64_t kWaitLimitNs3 = 2000000000ull;

template <typename T> struct Geom3 {
    static constexpr int HX = 16 / (int)sizeof(T);
    static constexpr int W = 58;
    // lanes read box columns shift .. shift + 64 with shift < HX
    static constexpr int BX = 64 + HX;
    __host__ __device__ static constexpr int box_x(int x0) { return (x0 - 4) & ~(HX - 1); }
    static constexpr int IBX = 80;   // 64 ids from at most 15 bytes into the id box
};

struct Fused3Params {
    const TileRec *recs;
    int ntiles;
    int parity;
    int *status;
    int stages;
    int slot_bytes;
    const int *first;   // per-CTA tile ranges (NULL: round-robin)
};

__host__ __device__ constexpr int al3(int v, int a) { return (v + a - 1) / a * a; }

template <typename T, int TY> __host__ __device__ constexpr int box3_bytes() {
    return Geom3<T>::BX * (TY + 6) * (int)sizeof(T);
}
template <typename T, int TY> __host__ __device__ constexpr int idbox3_off() { return al3(6 * box3_bytes<T, TY>(), 128); }
template <int TY> __host__ __device__ constexpr int idbox3_bytes() { return Geom3<float>::IBX * (TY + 6); }
template <typename T, int TY> __host__ __device__ constexpr int slot3_bytes() {
    return al3(idbox3_off<T, TY>() + idbox3_bytes<TY>(), 128);
}
constexpr int PW3 = 68;   // shared plane row pitch: column x - x0 + 4 (lane cells at 2 lane, + 1)
template <int TY> __host__ __device__ constexpr int PR3() { return TY + 7; }   // rows r + 1 for r in -1 .. TY+5
template <int TY> __host__ __device__ constexpr int plane3_floats() { return PR3<TY>() * PW3; }
constexpr int NPL3 = 14;   // H1, H2, H3 (Hx, Hz) | E1, E2 (Ex, Ez) x 2 buffers
constexpr int TAB3_BYTES = kMaxTable * 2 * 16;
template <typename T, int TY> __host__ __device__ constexpr int smem3_bytes(int stages) {
    return 256 + NTR3 * (int)sizeof(TileRec) + TAB3_BYTES + al3(NPL3 * plane3_floats<TY>() * 4, 128) +
           stages * slot3_bytes<T, TY>();
}
template <int TY> __host__ __device__ constexpr int threads3() { return (TY + 6) * 32; }

template <typename T, int TY>
__global__ void __launch_bounds__(threads3<TY>(), 1) fused3_step_kernel(const Fused3Params P) {
    using G = Geom3<T>;
    constexpr int BX = G::BX, W = G::W;
    constexpr int FB = box3_bytes<T, TY>(), FE = FB / (int)sizeof(T), IDO = idbox3_off<T, TY>();
    static_assert(FB % 16 == 0 && FE % 2 == 0, "field boxes keep 16-byte rows and even-aligned pairs");
    constexpr int NCW = TY + 5, NCT = NCW * 32;
    constexpr int PF = plane3_floats<TY>();

    extern __shared__ __align__(128) unsigned char smem[];
    if (smem_u32(smem) & 127u) {
        if (threadIdx.x == 0) atomicOr(P.status, STATUS_BADINDEX);
        return;
    }
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 8;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 128);
    TileRec *recs = reinterpret_cast<TileRec *>(smem + 256);
    float4 *stab = reinterpret_cast<float4 *>(smem + 256 + NTR3 * sizeof(TileRec));
    float *planes = reinterpret_cast<float *>(smem + 256 + NTR3 * sizeof(TileRec) + TAB3_BYTES);
    float *sh1x = planes, *sh1z = planes + PF, *sh2x = planes + 2 * PF, *sh2z = planes + 3 * PF;
    float *sh3x = planes + 4 * PF, *sh3z = planes + 5 * PF;
    float *e1b = planes + 6 * PF;    // [buffer][Ex, Ez][PF]
    float *e2b = planes + 10 * PF;   // [buffer][Ex, Ez][PF]
    unsigned char *slots = smem + 256 + NTR3 * sizeof(TileRec) + TAB3_BYTES + al3(NPL3 * PF * 4, 128);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = P.stages, SB = P.slot_bytes;
    const int t_begin = P.first ? __ldg(P.first + blockIdx.x) : (int)blockIdx.x;
    const int t_end = P.first ? __ldg(P.first + blockIdx.x + 1) : P.ntiles;
    const int t_step = P.first ? 1 : (int)gridDim.x;

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
    if (warp == NCW) {
        int issued = 0, m = 0, s = 0;
        uint32_t rnd = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; t += t_step) {
            TileRec *rec = &recs[m++ % NTR3];
            int kb = 0, klast = 0;
            for (int k = 0;; ++k) {
                if (issued >= S) {
                    const bool w = mbar_wait_abortable(&empty[s], rnd ^ 1u, kWaitLimitNs3, abort_flag, 0);
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
                    kb = rec->kz0 > 3 ? rec->kz0 - 3 : 0;
                    klast = rec->kz1 + 2;
                }
                const int kk = kb + k;
                if (lane == 0) {
                    const int src_copy = P.parity ^ rec->parity_off;
                    const bool has_id = rec->mode == COEF_ID8;
                    unsigned char *dst = slots + s * SB;
                    fence_proxy_async_smem();
                    if (tma_x_ok(P.status, G::box_x(rec->x0), (int)sizeof(T)) &&
                        (!has_id || tma_x_ok(P.status, rec->id_x0, 1))) {
                        mbar_arrive_expect_tx(&full[s], 6 * FB + (has_id ? idbox3_bytes<TY>() : 0));
                        tma_load_4d(dst, rec->maps + src_copy * 6, G::box_x(rec->x0), rec->y0 - 3, kk, 0, &full[s]);
                        if (has_id) tma_load_3d(dst + IDO, rec->maps + 12, rec->id_x0, rec->y0 - 3, kk, &full[s]);
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
                if (kk >= klast) break;
            }
        }
        if (!ok && lane == 0) {
            atomicOr(P.status, STATUS_TIMEOUT);
            for (int u = issued > S ? issued - S : 0; u < issued; ++u)
                mbar_wait_bounded(&full[u % S], (u / S) & 1, kWaitLimitNs3);
        }
        return;
    }

    // =========================================================== consumer warps
    const int r = warp;                      // row warp: y = y0 - 3 + r
    const int by = r;                        // box row
    const int pc = 2 * lane;                 // shared plane column of the first cell
    const int pr = r + 1;                    // shared plane row
    int sa = 0, m = 0;
    uint32_t pa = 0;
    const float4 *tab_cached = nullptr;
    auto wait_full = [&](int slot, uint32_t par) {
        return mbar_wait_abortable(&full[slot], par, kWaitLimitNs3, abort_flag, 0);
    };
    const float2 zero2 = make_float2(0.f, 0.f);

    for (int t = t_begin; t < t_end; t += t_step) {
        bool ok = wait_full(sa, pa);
        if (bar_sync_or(2, NCT, !ok || *abort_flag != 0)) {
            if (threadIdx.x == 0) atomicOr(P.status, STATUS_TIMEOUT);
            return;
        }
        const TileRec *rec = &recs[m++ % NTR3];
        const int x0 = rec->x0, y0 = rec->y0, kz0 = rec->kz0, kz1 = rec->kz1;
        const int bx = (x0 - 4) - G::box_x(x0) + 2 * lane;   // box column of the lane's first cell
        const int nx = rec->nx, ny = rec->ny, nz = rec->nz;
        const long long pitch = rec->pitch, plane = rec->plane;
        const bool id_mode = rec->mode == COEF_ID8;
        const bool ch_uni = rec->ch_uniform != 0;
        const int idoff = x0 - 4 - rec->id_x0;   // lane cells start this many bytes into the id box
        if (id_mode && rec->table != tab_cached) {
            const float4 *src = rec->table;
            const int n = 2 * rec->ntab;
            for (int e = threadIdx.x; e < n; e += NCT) stab[e] = __ldg(src + e);
            bar_sync_or(2, NCT, false);
            tab_cached = src;
        }
        const int dstc = (P.parity ^ rec->parity_off) ^ 1;
        T *const dst0 = static_cast<T *>(rec->dst[dstc][0]);   // the six arrays lie plane * nz apart
        const long long fstride = plane * nz;
        const float4 ce_s = make_float4(rec->ce[0], rec->ce[1], rec->ce[2], 0.f);
        const float4 ch_s = make_float4(rec->ch[0], rec->ch[1], rec->ch[2], 0.f);
        const int gj = y0 - 3 + r;
        const int gi = x0 - 4 + 2 * lane;       // first cell; second is gi + 1 (odd, never 0)
        const bool rowin = gj >= 0 && gj < ny;
        const bool ina = gi >= 0 && gi < nx, inb = gi + 1 >= 0 && gi + 1 < nx;
        const bool out_row = r >= 3 && r < TY + 3 && gj < ny;           // level-3 outputs of this row are stored
        const bool out_a = lane >= 2 && 2 * lane - 4 < W && gi < nx;   // both cells share the column window
        const int kb = kz0 > 3 ? kz0 - 3 : 0;
        const bool j1 = gj >= 1, i1a = gi >= 1;

        auto at = [&](const T *base, int f, int xx, int yy) { return base + f * FE + yy * BX + xx; };
        auto coef = [&](uint32_t ip, int which, float4 &a, float4 &b) {   // which: 0 ce, 1 ch
            if (id_mode && !(which && ch_uni)) {
                a = stab[2 * (ip & 0xff) + which];
                b = stab[2 * (ip >> 8) + which];
            } else {
                a = b = which ? ch_s : ce_s;
            }
        };
        // E update of one level (masked coefficients: tangential E at the faces i = 0, j = 0, k = 0 keeps
        // its value), in the operation order of every other kernel
        auto e_update = [&](uint32_t ip, int kp, float2 hx, float2 hy, float2 hz, float2 hx_ym, float2 hz_ym,
                            float hz_xm, float hy_xm, float2 hxp, float2 hyp, float2 ex, float2 ey, float2 ez,
                            float2 &ox, float2 &oy, float2 &oz) {
            float4 ca, cb;
            coef(ip, 0, ca, cb);
            const bool k1 = kp >= 1;
            const float2 cex = make_float2((j1 && k1) ? ca.x : 0.f, (j1 && k1) ? cb.x : 0.f);
            const float2 cey = make_float2((i1a && k1) ? ca.y : 0.f, k1 ? cb.y : 0.f);
            const float2 cez = make_float2((i1a && j1) ? ca.z : 0.f, j1 ? cb.z : 0.f);
            ox = fma2(cex, sub2(sub2(hz, hz_ym), sub2(hy, hyp)), ex);
            oy = fma2(cey, sub2(sub2(hx, hxp), sub2(hz, make_float2(hz_xm, hz.x))), ey);
            oz = fma2(cez, sub2(sub2(hy, make_float2(hy_xm, hy.x)), sub2(hx, hx_ym)), ez);
        };
        // H update of one level from E at this plane (own, z + 1, y + 1 row, x + 1 neighbour)
        auto h_update = [&](uint32_t ip, float2 ex, float2 ey, float2 ez, float2 exz, float2 eyz, float2 ex_y1,
                            float2 ez_y1, float ey_x2, float ez_x2, float2 hx, float2 hy, float2 hz, float2 &ox,
                            float2 &oy, float2 &oz) {
            float4 ca, cb;
            coef(ip, 1, ca, cb);
            const float2 ez_x1 = make_float2(ez.y, ez_x2), ey_x1 = make_float2(ey.y, ey_x2);
            ox = fma2(make_float2(ca.x, cb.x), sub2(sub2(eyz, ey), sub2(ez_y1, ez)), hx);
            oy = fma2(make_float2(ca.y, cb.y), sub2(sub2(ez_x1, ez), sub2(exz, ex)), hy);
            oz = fma2(make_float2(ca.z, cb.z), sub2(sub2(ex_y1, ex), sub2(ey_x1, ey)), hz);
        };

        float2 h1px = zero2, h1py = zero2, h1pz = zero2;   // H1(k-1)
        float2 e1px = zero2, e1py = zero2, e1pz = zero2;   // E1(k-1)
        float2 h2px = zero2, h2py = zero2, h2pz = zero2;   // H2(k-2)
        float2 e2px = zero2, e2py = zero2, e2pz = zero2;   // E2(k-2)
        float2 h3px = zero2, h3py = zero2;                 // H3(k-3) (Hx, Hy)
        uint32_t id1 = 0, id2 = 0;                          // material ids of planes k-1 and k-2

        for (int k = kb; k <= kz1 + 1; ++k) {
            int sb = sa + 1;
            uint32_t pb = pa;
            if (sb == S) {
                sb = 0;
                pb ^= 1u;
            }
            ok = wait_full(sb, pb);
            ok = __all_sync(0xffffffffu, ok);
            const T *A = reinterpret_cast<const T *>(slots + sa * SB);
            const T *B = reinterpret_cast<const T *>(slots + sb * SB);
            const uint8_t *ida = slots + sa * SB + IDO;
            // level l runs on plane k - l + 1 from k >= kz0 - 3 + 2l - 2 (H) and kz0 - 3 + 2l - 1 (E), and never
            // below plane 0; level 3's E is stored for planes kz0 .. kz1 - 1
            const bool do_e1 = k >= kz0 - 2;
            const bool do_h2 = k >= kz0 - 1 && k >= 1, do_e2 = k >= kz0 && k >= 1;
            const bool do_h3 = k >= kz0 + 1 && k >= 2, do_e3 = k >= kz0 + 2;
            float *e1cur = e1b + (k & 1) * 2 * PF, *e1prv = e1b + ((k + 1) & 1) * 2 * PF;
            float *e2cur = e2b + (k & 1) * 2 * PF, *e2prv = e2b + ((k + 1) & 1) * 2 * PF;

            // ---------------- H1(k)
            float2 e0x = zero2, e0y = zero2, e0z = zero2, h1x = zero2, h1y = zero2, h1z = zero2;
            uint32_t id0 = 0;
            if (ok) {
                e0x = Pair<T>::ld(at(A, 0, bx, by));
                e0y = Pair<T>::ld(at(A, 1, bx, by));
                e0z = Pair<T>::ld(at(A, 2, bx, by));
                const float2 ex_y1 = Pair<T>::ld(at(A, 0, bx, by + 1));
                const float2 ez_y1 = Pair<T>::ld(at(A, 2, bx, by + 1));
                const float ey_x2 = Pair<T>::ld1(at(A, 1, bx + 2, by));
                const float ez_x2 = Pair<T>::ld1(at(A, 2, bx + 2, by));
                const float2 exb = Pair<T>::ld(at(B, 0, bx, by));
                const float2 eyb = Pair<T>::ld(at(B, 1, bx, by));
                const float2 hx0 = Pair<T>::ld(at(A, 3, bx, by));
                const float2 hy0 = Pair<T>::ld(at(A, 4, bx, by));
                const float2 hz0 = Pair<T>::ld(at(A, 5, bx, by));
                if (id_mode) id0 = *reinterpret_cast<const uint16_t *>(ida + by * G::IBX + idoff + 2 * lane);
                h_update(id0, e0x, e0y, e0z, exb, eyb, ex_y1, ez_y1, ey_x2, ez_x2, hx0, hy0, hz0, h1x, h1y, h1z);
                *reinterpret_cast<float2 *>(sh1x + pr * PW3 + pc) = h1x;
                *reinterpret_cast<float2 *>(sh1z + pr * PW3 + pc) = h1z;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(NCT) : "memory");

            // ---------------- E1(k), zero outside the cavity
            float2 e1x = zero2, e1y = zero2, e1z = zero2;
            if (ok && do_e1 && r >= 1) {
                const float2 hx_ym = *reinterpret_cast<const float2 *>(sh1x + (pr - 1) * PW3 + pc);
                const float2 hz_ym = *reinterpret_cast<const float2 *>(sh1z + (pr - 1) * PW3 + pc);
                const float hz_xm = __shfl_up_sync(0xffffffffu, h1z.y, 1);
                const float hy_xm = __shfl_up_sync(0xffffffffu, h1y.y, 1);
                e_update(id0, k, h1x, h1y, h1z, hx_ym, hz_ym, hz_xm, hy_xm, h1px, h1py, e0x, e0y, e0z, e1x, e1y, e1z);
                const bool inz = k < nz;
                if (!(rowin && ina && inz)) e1x.x = e1y.x = e1z.x = 0.f;
                if (!(rowin && inb && inz)) e1x.y = e1y.y = e1z.y = 0.f;
                *reinterpret_cast<float2 *>(e1cur + pr * PW3 + pc) = e1x;
                *reinterpret_cast<float2 *>(e1cur + PF + pr * PW3 + pc) = e1z;
            }
            // ---------------- H2(k-1) = H1(k-1) - ch curl E1 (z + 1 from plane k, y + 1 from the row below's
            // E1(k-1), written the iteration before)
            float2 h2x = zero2, h2y = zero2, h2z = zero2;
            if (ok && do_h2 && r >= 1 && r <= TY + 3) {
                const float2 ex_y1 = *reinterpret_cast<const float2 *>(e1prv + (pr + 1) * PW3 + pc);
                const float2 ez_y1 = *reinterpret_cast<const float2 *>(e1prv + PF + (pr + 1) * PW3 + pc);
                const float ey_x2 = __shfl_down_sync(0xffffffffu, e1py.x, 1);
                const float ez_x2 = __shfl_down_sync(0xffffffffu, e1pz.x, 1);
                h_update(id1, e1px, e1py, e1pz, e1x, e1y, ex_y1, ez_y1, ey_x2, ez_x2, h1px, h1py, h1pz, h2x, h2y, h2z);
                *reinterpret_cast<float2 *>(sh2x + pr * PW3 + pc) = h2x;
                *reinterpret_cast<float2 *>(sh2z + pr * PW3 + pc) = h2z;
            }
            const float h2z_xm = __shfl_up_sync(0xffffffffu, h2z.y, 1);
            const float h2y_xm = __shfl_up_sync(0xffffffffu, h2y.y, 1);
            asm volatile("bar.sync 1, %0;" ::"r"(NCT) : "memory");

            // ---------------- E2(k-1), zero outside the cavity
            float2 e2x = zero2, e2y = zero2, e2z = zero2;
            if (ok && do_e2 && r >= 2 && r <= TY + 3) {
                const float2 hx_ym = *reinterpret_cast<const float2 *>(sh2x + (pr - 1) * PW3 + pc);
                const float2 hz_ym = *reinterpret_cast<const float2 *>(sh2z + (pr - 1) * PW3 + pc);
                e_update(id1, k - 1, h2x, h2y, h2z, hx_ym, hz_ym, h2z_xm, h2y_xm, h2px, h2py, e1px, e1py, e1pz, e2x,
                         e2y, e2z);
                const bool inz = k - 1 < nz;
                if (!(rowin && ina && inz)) e2x.x = e2y.x = e2z.x = 0.f;
                if (!(rowin && inb && inz)) e2x.y = e2y.y = e2z.y = 0.f;
                *reinterpret_cast<float2 *>(e2cur + pr * PW3 + pc) = e2x;
                *reinterpret_cast<float2 *>(e2cur + PF + pr * PW3 + pc) = e2z;
            }
            // ---------------- H3(k-2) = H2(k-2) - ch curl E2 (z + 1 from plane k-1, y + 1 from the row below's
            // E2(k-2), written the iteration before)
            float2 h3x = zero2, h3y = zero2, h3z = zero2;
            if (ok && do_h3 && r >= 2 && r <= TY + 2) {
                const float2 ex_y1 = *reinterpret_cast<const float2 *>(e2prv + (pr + 1) * PW3 + pc);
                const float2 ez_y1 = *reinterpret_cast<const float2 *>(e2prv + PF + (pr + 1) * PW3 + pc);
                const float ey_x2 = __shfl_down_sync(0xffffffffu, e2py.x, 1);
                const float ez_x2 = __shfl_down_sync(0xffffffffu, e2pz.x, 1);
                h_update(id2, e2px, e2py, e2pz, e2x, e2y, ex_y1, ez_y1, ey_x2, ez_x2, h2px, h2py, h2pz, h3x, h3y, h3z);
                *reinterpret_cast<float2 *>(sh3x + pr * PW3 + pc) = h3x;
                *reinterpret_cast<float2 *>(sh3z + pr * PW3 + pc) = h3z;
            }
            const float h3z_xm = __shfl_up_sync(0xffffffffu, h3z.y, 1);
            const float h3y_xm = __shfl_up_sync(0xffffffffu, h3y.y, 1);
            asm volatile("bar.sync 1, %0;" ::"r"(NCT) : "memory");

            // ---------------- E3(k-2) and the level-3 stores
            if (ok && do_e3 && out_row) {
                const float2 hx_ym = *reinterpret_cast<const float2 *>(sh3x + (pr - 1) * PW3 + pc);
                const float2 hz_ym = *reinterpret_cast<const float2 *>(sh3z + (pr - 1) * PW3 + pc);
                float2 e3x, e3y, e3z;
                e_update(id2, k - 2, h3x, h3y, h3z, hx_ym, hz_ym, h3z_xm, h3y_xm, h3px, h3py, e2px, e2py, e2pz, e3x,
                         e3y, e3z);
                const long long g = (long long)(k - 2) * plane + (long long)gj * pitch + gi;
                if (out_a && store_ok(P.status, g, 2, plane * nz)) {
                    Pair<T>::st_cs(dst0 + g, e3x.x, e3x.y);
                    Pair<T>::st_cs(dst0 + g + 1 * fstride, e3y.x, e3y.y);
                    Pair<T>::st_cs(dst0 + g + 2 * fstride, e3z.x, e3z.y);
                    Pair<T>::st_cs(dst0 + g + 3 * fstride, h3x.x, h3x.y);
                    Pair<T>::st_cs(dst0 + g + 4 * fstride, h3y.x, h3y.y);
                    Pair<T>::st_cs(dst0 + g + 5 * fstride, h3z.x, h3z.y);
                }
            }
            // ---------------- carry the z neighbours to the next plane
            h3px = h3x;
            h3py = h3y;
            h2px = h2x;
            h2py = h2y;
            h2pz = h2z;
            e2px = e2x;
            e2py = e2y;
            e2pz = e2z;
            h1px = h1x;
            h1py = h1y;
            h1pz = h1z;
            e1px = e1x;
            e1py = e1y;
            e1pz = e1z;
            id2 = id1;
            id1 = id0;
            // ---------------- release unit k (and k+1 after the last plane)
            const bool last = k == kz1 + 1;
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

template <typename T, int TY>
cudaError_t launch3_typed(const FusedLaunch &L, cudaStream_t s) {
    const int smem = smem3_bytes<T, TY>(L.stages);
    auto kern = fused3_step_kernel<T, TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    Fused3Params P;
    P.recs = L.recs;
    P.ntiles = L.ntiles;
    P.parity = L.parity;
    P.status = L.status;
    P.stages = L.stages;
    P.slot_bytes = slot3_bytes<T, TY>();
    P.first = L.first;
    kern<<<L.grid, threads3<TY>(), smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T, int TY>
cudaError_t occupancy3_typed(int stages, int *n) {
    const int smem = smem3_bytes<T, TY>(stages);
    auto kern = fused3_step_kernel<T, TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, threads3<TY>(), smem);
}

#define FDTD_DISPATCH3(storage, tile_y, ...)                                                          \
    do {                                                                                              \
        if (storage == 0) {                                                                           \
            if (tile_y == 8) { using T = float; constexpr int TY = 8; __VA_ARGS__; }                  \
            else if (tile_y == 10) { using T = float; constexpr int TY = 10; __VA_ARGS__; }           \
            else if (tile_y == 12) { using T = float; constexpr int TY = 12; __VA_ARGS__; }           \
        } else if (storage == 1) {                                                                    \
            if (tile_y == 8) { using T = __half; constexpr int TY = 8; __VA_ARGS__; }                 \
            else if (tile_y == 10) { using T = __half; constexpr int TY = 10; __VA_ARGS__; }          \
            else if (tile_y == 12) { using T = __half; constexpr int TY = 12; __VA_ARGS__; }          \
        } else if (storage == 2) {                                                                    \
            if (tile_y == 8) { using T = __nv_bfloat16; constexpr int TY = 8; __VA_ARGS__; }          \
            else if (tile_y == 10) { using T = __nv_bfloat16; constexpr int TY = 10; __VA_ARGS__; }   \
            else if (tile_y == 12) { using T = __nv_bfloat16; constexpr int TY = 12; __VA_ARGS__; }   \
        }                                                                                             \
    } while (0)

}  // namespace

int fused3_tile_w() { return Geom3<float>::W; }

int fused3_smem_bytes(int storage, int tile_y, int stages) {
    int r = -1;
    FDTD_DISPATCH3(storage, tile_y, r = smem3_bytes<T, TY>(stages));
    return r;
}

cudaError_t fused3_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm) {
    cudaError_t e = cudaErrorInvalidValue;
    FDTD_DISPATCH3(storage, tile_y, e = occupancy3_typed<T, TY>(stages, ctas_per_sm));
    return e;
}

cudaError_t launch_fused3_step(int storage, const FusedLaunch &L, cudaStream_t s) {
    if (L.ntiles <= 0) return cudaSuccess;
    if (L.stages < 3 || L.stages > 8 || L.step) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    FDTD_DISPATCH3(storage, L.tile_y, e = (launch3_typed<T, TY>(L, s)));
    return e;
}

}  // namespace fdtd
