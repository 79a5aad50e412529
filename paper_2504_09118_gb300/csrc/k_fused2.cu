// Two Yee leapfrog steps per pass over HBM (temporal blocking, T = 2) for sm_103a.
//
// Same update as k_fused.cu (Eq. 2 of the paper in the order of Listing 1, PEC by
// index predicates), applied twice per launch: level 1 takes (H^{n-1/2}, E^n) to
// (H^{n+1/2}, E^{n+1}) and level 2 takes that to (H^{n+3/2}, E^{n+2}); only level 2
// is written to HBM (copy 1-s), so a step costs half the DRAM bytes of the one-step
// kernel at the price of recomputing a wider halo.
//
// Tile: W = 60 output columns x TY output rows, over planes [kz0, kz1); the TMA box starts at
// x0 - 2 rounded down to the 16-byte granule (Geom2::box_x).  Consumer warps
// r = 0..TY+2 own rows y = y0 - 2 + r; each lane owns the two cells x0 - 2 + 2 lane,
// +1, so the lanes cover [x0 - 2, x0 + 62) at both levels:
//   level 1  H1 rows y0-2 .. y0+TY,   E1 rows y0-1 .. y0+TY    (from units k, k+1)
//   level 2  H2 rows y0-1 .. y0+TY-1, E2 rows y0 .. y0+TY-1    (one plane behind)
// which is exactly what the outputs need (a stored value never depends on a lane's
// unused edge cells).  E1 outside the cavity is forced to 0: at i = nx, j = ny or k = nz
// it is tangential to a PEC face.  x neighbours come from lane shuffles, y neighbours
// from small shared planes (H1 and H2: Hx, Hz of the row above; E1: Ex, Ez of the row
// below, double-buffered in z); z neighbours stay in registers.
//
// Per z-plane iteration j: [H1(j)] bar [E1(j)] [H2(j-1)] bar [E2(j-1) + stores], the last phase
// running into the next plane's H1 (they share no data); H2(j-1) reads no E1(j) of another warp, so
// E1 and H2 need no barrier between them.  A producer warp streams plane units (six field boxes with
// a 2-cell halo in y, id box) through an S-slot TMA ring exactly as the one-step kernel does; waits
// are bounded and a shared abort flag ends the CTA together (see k_fused.cu).
//
// The plane iteration is one body compiled twice.  The general instance tests, per plane, which
// phases run and which PEC masks apply (a tile's first planes and its last one); the steady instance
// runs the planes in between, where neither depends on the plane.  With PEC-coded material ids (the
// faces a cell lies on select a table entry whose tangential E coefficients are zero, and entry 0,
// read outside the cavity, has ce = 0) the steady planes apply no masks at all.  Every value keeps
// the operation sequence of the one-step kernel: a masked coefficient there is the same zero in the
// same fused multiply-add.  The kernel is compiled per coefficient class (CoefClass), so a single
// cavity's launch tests its coefficient layout nowhere; batches keep a runtime class and the general
// body.
#include <type_traits>

#include "fused_common.cuh"
#include "launch.h"

namespace fdtd {

namespace {

using namespace fused;

constexpr int NTR2 = 8;
constexpr uint64_t kWaitLimitNs2 = 2000000000ull;

template <typename T> struct Geom2 {
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

struct Fused2Params {
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

__host__ __device__ constexpr int al(int v, int a) { return (v + a - 1) / a * a; }

template <typename T, int TY> __host__ __device__ constexpr int box_bytes() {
    return Geom2<T>::BX * (TY + 4) * (int)sizeof(T);
}
// The 4-D load lands the six field boxes back to back (field stride = box bytes, a multiple of 16); the id
// box, a load of its own, starts at the next 128-byte boundary.
template <typename T, int TY> __host__ __device__ constexpr int idbox_off() { return al(6 * box_bytes<T, TY>(), 128); }
template <int TY> __host__ __device__ constexpr int idbox_bytes() { return Geom2<float>::IBX * (TY + 4); }
template <typename T, int TY> __host__ __device__ constexpr int slot2_bytes() {
    return al(idbox_off<T, TY>() + idbox_bytes<TY>(), 128);
}
constexpr int PW = 68;   // shared plane row pitch: column x - x0 + 4 (lane cells at 2 lane + 2, + 3)
template <int TY> __host__ __device__ constexpr int PR() { return TY + 5; }   // rows: r + 1 for r in -1 .. TY+3
template <int TY> __host__ __device__ constexpr int plane_floats() { return PR<TY>() * PW; }
constexpr int TAB2_BYTES = kMaxTable * 2 * 16;
template <typename T, int TY> __host__ __device__ constexpr int smem2_bytes(int stages) {
    // barriers/abort | records | table | H1 (Hx,Hz) | H2 (Hx,Hz) | E1 (Ex,Ez) x 2 | ring
    return 256 + NTR2 * (int)sizeof(TileRec) + TAB2_BYTES + al(8 * plane_floats<TY>() * 4, 128) +
           stages * slot2_bytes<T, TY>();
}
template <int TY> __host__ __device__ constexpr int threads2() { return (TY + 4) * 32; }

// BATCH: tiles carry their member's stop clock (skip finished members, one-step stores for a member
// with one step left); a single cavity's launch compiles without those checks.  CM: the CoefClass of
// every tile (COEF_CLASS_ANY reads each record's mode), so that a single cavity's kernel carries no
// per-plane test of its coefficient layout.
template <typename T, int TY, bool BATCH, int CM>
__global__ void __launch_bounds__(threads2<TY>(), 1) fused2_step_kernel(const Fused2Params P) {
    using G = Geom2<T>;
    constexpr int BX = G::BX, W = G::W;
    constexpr int FB = box_bytes<T, TY>(), FE = FB / (int)sizeof(T), IDO = idbox_off<T, TY>();
    static_assert(FB % 16 == 0 && FE % 2 == 0, "field boxes keep 16-byte rows and even-aligned pairs");
    constexpr int NCW = TY + 3, NCT = NCW * 32;
    constexpr int PF = plane_floats<TY>();
    // the steady-state plane body (below) for launches of one coefficient layout; a batch, whose
    // instance also carries the stop-clock logic, runs every plane through the general body, which
    // needs fewer registers (no spill at 16 rows)
    constexpr bool SPLIT = !BATCH && CM != COEF_CLASS_ANY;
    // PEC-coded ids (COEF_CLASS_PEC_*): the table zeroes the E coefficients on the faces and outside the
    // cavity (where the box read E = 0, so fma(0, curl, 0) = +0), so the steady planes need no masks
    constexpr bool PEC_TABLE = CM == COEF_CLASS_PEC_ID_UNIFORM_H || CM == COEF_CLASS_PEC_ID;

    extern __shared__ __align__(128) unsigned char smem[];
    if (smem_u32(smem) & 127u) {
        if (threadIdx.x == 0) atomicOr(P.status, STATUS_BADINDEX);
        return;
    }
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 8;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 128);
    TileRec *recs = reinterpret_cast<TileRec *>(smem + 256);
    float4 *stab = reinterpret_cast<float4 *>(smem + 256 + NTR2 * sizeof(TileRec));
    float *planes = reinterpret_cast<float *>(smem + 256 + NTR2 * sizeof(TileRec) + TAB2_BYTES);
    float *sh1x = planes, *sh1z = planes + PF, *sh2x = planes + 2 * PF, *sh2z = planes + 3 * PF;
    float *e1b = planes + 4 * PF;   // [buffer][Ex, Ez][PF]
    unsigned char *slots = smem + 256 + NTR2 * sizeof(TileRec) + TAB2_BYTES + al(8 * PF * 4, 128);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = P.stages, SB = P.slot_bytes;
    // this CTA's tiles: a host-balanced contiguous range, or every gridDim.x-th tile
    const int t_begin = P.first ? __ldg(P.first + blockIdx.x) : (int)blockIdx.x;
    const int t_end = P.first ? __ldg(P.first + blockIdx.x + 1) : P.ntiles;
    const int t_step = P.first ? 1 : (int)gridDim.x;
    // Steps a tile takes in this launch: min(launch_steps, stop - clock); a batch member with one step
    // left stores its level-1 result, a finished member's tiles are skipped (producer and consumers alike).
    const long long clock = BATCH ? *P.step : 0;

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
            if (BATCH && __ldg(&P.recs[t].stop) <= clock) continue;   // member already took its last step
            TileRec *rec = &recs[m++ % NTR2];
            int kb = 0, klast = 0;
            for (int k = 0;; ++k) {
                if (issued >= S) {
                    const bool w = mbar_wait_abortable(&empty[s], rnd ^ 1u, kWaitLimitNs2, abort_flag, 0);
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
                    const bool has_id = CM == COEF_CLASS_ANY ? rec->mode == COEF_ID8 : CM >= COEF_CLASS_ID_UNIFORM_H;
                    unsigned char *dst = slots + s * SB;
                    fence_proxy_async_smem();
                    if (tma_x_ok(P.status, G::box_x(rec->x0), (int)sizeof(T)) &&
                        (!has_id || tma_x_ok(P.status, rec->id_x0, 1))) {
                        mbar_arrive_expect_tx(&full[s], 6 * FB + (has_id ? idbox_bytes<TY>() : 0));
                        // the six field boxes in one load: a 4-D box (x, y, plane, field) lands as six
                        // consecutive FB-byte boxes
                        tma_load_4d(dst, rec->maps + src_copy * 6, G::box_x(rec->x0), rec->y0 - 2, kk, 0, &full[s]);
                        if (has_id)
                            tma_load_3d(dst + IDO, rec->maps + 12, rec->id_x0, rec->y0 - 2, kk, &full[s]);
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
                mbar_wait_bounded(&full[u % S], (u / S) & 1, kWaitLimitNs2);
        }
        return;
    }

    // =========================================================== consumer warps
    const int r = warp;                      // row warp: y = y0 - 2 + r
    const int by = r;                        // box row
    const int pc = 2 * lane + 2;             // shared plane column of the first cell
    const int pr = r + 1;                    // shared plane row
    int sa = 0, m = 0;
    uint32_t pa = 0;
    const float4 *tab_cached = nullptr;
    auto wait_full = [&](int slot, uint32_t par) {
        return mbar_wait_abortable(&full[slot], par, kWaitLimitNs2, abort_flag, 0);
    };
    const float2 zero2 = make_float2(0.f, 0.f);

    for (int t = t_begin; t < t_end; t += t_step) {
        if (BATCH && __ldg(&P.recs[t].stop) <= clock) continue;   // same skip rule as the producer
        bool ok0 = wait_full(sa, pa);
        if (bar_sync_or(2, NCT, !ok0 || *abort_flag != 0)) {
            if (threadIdx.x == 0) atomicOr(P.status, STATUS_TIMEOUT);
            return;
        }
        const TileRec *rec = &recs[m++ % NTR2];
        const int x0 = rec->x0, y0 = rec->y0, kz0 = rec->kz0, kz1 = rec->kz1;
        const int bx = (x0 - 2) - G::box_x(x0) + 2 * lane;   // box column of the lane's first cell
        const int nx = rec->nx, ny = rec->ny, nz = rec->nz;
        const long long pitch = rec->pitch, plane = rec->plane;
        const bool id_mode = CM == COEF_CLASS_ANY ? rec->mode == COEF_ID8 : CM >= COEF_CLASS_ID_UNIFORM_H;
        const bool ch_uni = CM == COEF_CLASS_ANY ? rec->ch_uniform != 0 : CM != COEF_CLASS_ID && CM != COEF_CLASS_PEC_ID;
        const int idoff = x0 - 2 - rec->id_x0;   // lane cells start this many bytes into the id box
        if (id_mode && rec->table != tab_cached) {
            const float4 *src = rec->table;
            const int n = 2 * rec->ntab;
            for (int e = threadIdx.x; e < n; e += NCT) stab[e] = __ldg(src + e);
            bar_sync_or(2, NCT, false);
            tab_cached = src;
        }
        const int dstc = (P.parity ^ rec->parity_off) ^ 1;
        // the six arrays of a copy lie in one allocation, plane * nz elements apart: one base pointer
        // and a stride instead of six pointers (eight registers fewer)
        T *const dst0 = static_cast<T *>(rec->dst[dstc][0]);
        const long long fstride = plane * nz;
        const float4 ce_s = make_float4(rec->ce[0], rec->ce[1], rec->ce[2], 0.f);
        const float4 ch_s = make_float4(rec->ch[0], rec->ch[1], rec->ch[2], 0.f);
        const int gj = y0 - 2 + r;
        const int gi = x0 - 2 + 2 * lane;       // first cell; second is gi + 1
        const bool rowin = gj >= 0 && gj < ny;
        const bool ina = gi >= 0 && gi < nx, inb = gi + 1 < nx;   // gi + 1 >= 0 always for gi >= -2
        const bool out_row = r >= 2 && r < TY + 2 && gj < ny;      // level-2 outputs of this row are stored
        const bool out_a = lane >= 1 && 2 * lane - 2 < W && gi < nx; // both cells share the column window
        const int kb = kz0 > 2 ? kz0 - 2 : 0;
        // planes [ks, kz1) run every phase with no plane-dependent mask (k >= 1 for E1 and k - 1 >= 1 for
        // E2, k < nz, not the tile's last plane); the planes before ks and the last plane kz1 test them
        const int ks = kz0 + 1 > 2 ? kz0 + 1 : 2;
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
        float2 h1px = zero2, h1py = zero2, h1pz = zero2;   // H1(j-1) of own cells
        float2 e1px = zero2, e1py = zero2, e1pz = zero2;   // E1(j-1)
        float2 h2px = zero2, h2py = zero2;                 // H2(j-2) (Hx, Hy)
        uint32_t idprev = 0;                               // material ids of plane j-1

        // One z-plane iteration.  ST (steady): k in [ks, kz1), where every phase runs, no mask depends on
        // k, and a failed ring wait only drops the stores: the phases then read a stale slot (in bounds)
        // instead of being skipped, so nothing is zeroed or voted per plane.
        auto plane_step = [&](const int k, auto steady) {
            constexpr bool ST = decltype(steady)::value;
            int sb = sa + 1;
            uint32_t pb = pa;
            if (sb == S) {
                sb = 0;
                pb ^= 1u;
            }
            // unit k (slot sa) was waited for as the next unit of the previous plane, or at the tile start
            bool ok = wait_full(sb, pb);
            if (!ST) ok = __all_sync(0xffffffffu, ok);   // warp-uniform: the phases below shuffle across lanes
            const bool run = ST || ok;
            const T *A = reinterpret_cast<const T *>(slots + sa * SB);
            const T *B = reinterpret_cast<const T *>(slots + sb * SB);
            const uint8_t *ida = slots + sa * SB + IDO;
            // H2(k-1) needs plane k-1 >= 0 (its inputs at plane -1 were never written)
            const bool do_e1 = ST || k >= kz0 - 1;
            const bool do_h2 = !level1_only && (ST || (k >= kz0 && k >= 1));
            const bool do_e2 = !level1_only && (ST || k >= kz0 + 1);
            float *e1cur = e1b + (k & 1) * 2 * PF, *e1prv = e1b + ((k + 1) & 1) * 2 * PF;

            // ---------------- phase 1: H1(k) on the lane's two cells
            float2 e0x, e0y, e0z, h1x_, h1y_, h1z_;
            uint32_t idpair = 0;
            if (!ST) e0x = e0y = e0z = h1x_ = h1y_ = h1z_ = zero2;
            if (run) {
                e0x = Pair<T>::ld(at(A, 0, bx, by));
                e0y = Pair<T>::ld(at(A, 1, bx, by));
                e0z = Pair<T>::ld(at(A, 2, bx, by));
                const float2 ex_y1 = Pair<T>::ld(at(A, 0, bx, by + 1));
                const float2 ez_y1 = Pair<T>::ld(at(A, 2, bx, by + 1));
                const float ey_x2 = Pair<T>::ld1(at(A, 1, bx + 2, by));
                const float ez_x2 = Pair<T>::ld1(at(A, 2, bx + 2, by));
                const float2 exb = Pair<T>::ld(at(B, 0, bx, by));
                const float2 eyb = Pair<T>::ld(at(B, 1, bx, by));
                h1x_ = Pair<T>::ld(at(A, 3, bx, by));
                h1y_ = Pair<T>::ld(at(A, 4, bx, by));
                h1z_ = Pair<T>::ld(at(A, 5, bx, by));
                // idoff is even (x0 and the 16-byte id box origin are), so the lane's two ids are one aligned u16
                if (id_mode) idpair = *reinterpret_cast<const uint16_t *>(ida + by * G::IBX + idoff + 2 * lane);
                float4 ca, cb;
                coef(idpair, 1, ca, cb);
                const float2 ez_x1 = make_float2(e0z.y, ez_x2), ey_x1 = make_float2(e0y.y, ey_x2);
                h1x_ = fma2(make_float2(ca.x, cb.x), sub2(sub2(eyb, e0y), sub2(ez_y1, e0z)), h1x_);
                h1y_ = fma2(make_float2(ca.y, cb.y), sub2(sub2(ez_x1, e0z), sub2(exb, e0x)), h1y_);
                h1z_ = fma2(make_float2(ca.z, cb.z), sub2(sub2(ex_y1, e0x), sub2(ey_x1, e0y)), h1z_);
                *reinterpret_cast<float2 *>(sh1x + pr * PW + pc) = h1x_;
                *reinterpret_cast<float2 *>(sh1z + pr * PW + pc) = h1z_;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(NCT) : "memory");

            // ---------------- phase 2: E1(k) (zero outside the cavity: tangential at its far faces)
            // (in ST, a row that skips a phase leaves its pairs unset: no later phase of that row reads them)
            float2 e1x, e1y, e1z;
            if (!ST) e1x = e1y = e1z = zero2;
            if (run && do_e1 && r >= 1) {
                const float2 hx_ym = *reinterpret_cast<const float2 *>(sh1x + (pr - 1) * PW + pc);
                const float2 hz_ym = *reinterpret_cast<const float2 *>(sh1z + (pr - 1) * PW + pc);
                const float hz_xm = __shfl_up_sync(0xffffffffu, h1z_.y, 1);
                const float hy_xm = __shfl_up_sync(0xffffffffu, h1y_.y, 1);
                float4 ca, cb;
                coef(idpair, 0, ca, cb);
                const bool inz = ST || k < nz, k1 = ST || k >= 1, j1 = gj >= 1;
                const bool va = rowin && ina && inz, vb = rowin && inb && inz;
                const bool i1a = gi >= 1;
                constexpr bool NOMASK = ST && PEC_TABLE;
                const float2 cex = NOMASK ? make_float2(ca.x, cb.x)
                                          : make_float2((j1 && k1) ? ca.x : 0.f, (j1 && k1) ? cb.x : 0.f);
                const float2 cey = NOMASK ? make_float2(ca.y, cb.y)
                                          : make_float2((i1a && k1) ? ca.y : 0.f, k1 ? cb.y : 0.f);
                const float2 cez = NOMASK ? make_float2(ca.z, cb.z)
                                          : make_float2((i1a && j1) ? ca.z : 0.f, j1 ? cb.z : 0.f);
                e1x = fma2(cex, sub2(sub2(h1z_, hz_ym), sub2(h1y_, h1py)), e0x);
                e1y = fma2(cey, sub2(sub2(h1x_, h1px), sub2(h1z_, make_float2(hz_xm, h1z_.x))), e0y);
                e1z = fma2(cez, sub2(sub2(h1y_, make_float2(hy_xm, h1y_.x)), sub2(h1x_, hx_ym)), e0z);
                if (!NOMASK && !va) { e1x.x = 0.f; e1y.x = 0.f; e1z.x = 0.f; }
                if (!NOMASK && !vb) { e1x.y = 0.f; e1y.y = 0.f; e1z.y = 0.f; }
                *reinterpret_cast<float2 *>(e1cur + pr * PW + pc) = e1x;
                *reinterpret_cast<float2 *>(e1cur + PF + pr * PW + pc) = e1z;
                // one step: (H1, E1) is the result
                if (level1_only && ok && out_row && out_a && (ST || (k >= kz0 && k < kz1))) {
                    const long long g = (long long)k * plane + (long long)gj * pitch + gi;
                    if (store_ok(P.status, g, 2, plane * nz)) {
                        Pair<T>::st_cs(dst0 + g, e1x.x, e1x.y);
                        Pair<T>::st_cs(dst0 + g + 1 * fstride, e1y.x, e1y.y);
                        Pair<T>::st_cs(dst0 + g + 2 * fstride, e1z.x, e1z.y);
                        Pair<T>::st_cs(dst0 + g + 3 * fstride, h1x_.x, h1x_.y);
                        Pair<T>::st_cs(dst0 + g + 4 * fstride, h1y_.x, h1y_.y);
                        Pair<T>::st_cs(dst0 + g + 5 * fstride, h1z_.x, h1z_.y);
                    }
                }
            }
            // No barrier here: phase 3 reads only this lane's E1(k), its warp's E1(k-1) (shuffles) and the
            // row below's E1(k-1), written in the previous iteration (e1prv, the other buffer).  The
            // write-after-read hazards are covered by the remaining barriers: E1(k+1) overwrites e1prv's
            // buffer after the phase-3 -> 4 barrier of this iteration and the phase-1 -> 2 barrier of the next.

            // ---------------- phase 3: H2(k-1) = H1(k-1) - ch curl E1 (plane k-1, z+1 from plane k)
            float2 h2x, h2y, h2z;
            if (!ST) h2x = h2y = h2z = zero2;
            if (run && do_h2 && r >= 1 && r <= TY + 1) {
                const float2 ex_y1 = *reinterpret_cast<const float2 *>(e1prv + (pr + 1) * PW + pc);
                const float2 ez_y1 = *reinterpret_cast<const float2 *>(e1prv + PF + (pr + 1) * PW + pc);
                const float ey_x2 = __shfl_down_sync(0xffffffffu, e1py.x, 1);
                const float ez_x2 = __shfl_down_sync(0xffffffffu, e1pz.x, 1);
                float4 ca, cb;
                coef(idprev, 1, ca, cb);
                const float2 ez_x1 = make_float2(e1pz.y, ez_x2), ey_x1 = make_float2(e1py.y, ey_x2);
                h2x = fma2(make_float2(ca.x, cb.x), sub2(sub2(e1y, e1py), sub2(ez_y1, e1pz)), h1px);
                h2y = fma2(make_float2(ca.y, cb.y), sub2(sub2(ez_x1, e1pz), sub2(e1x, e1px)), h1py);
                h2z = fma2(make_float2(ca.z, cb.z), sub2(sub2(ex_y1, e1px), sub2(ey_x1, e1py)), h1pz);
                *reinterpret_cast<float2 *>(sh2x + pr * PW + pc) = h2x;
                *reinterpret_cast<float2 *>(sh2z + pr * PW + pc) = h2z;
            }
            // shuffles below are executed by whole warps; every lane takes part
            const float h2z_xm = __shfl_up_sync(0xffffffffu, h2z.y, 1);
            const float h2y_xm = __shfl_up_sync(0xffffffffu, h2y.y, 1);
            asm volatile("bar.sync 1, %0;" ::"r"(NCT) : "memory");

            // ---------------- phase 4: E2(k-1) = E1(k-1) + ce curl H2, and the level-2 stores
            if (run && do_e2 && out_row) {
                const float2 hx_ym = *reinterpret_cast<const float2 *>(sh2x + (pr - 1) * PW + pc);
                const float2 hz_ym = *reinterpret_cast<const float2 *>(sh2z + (pr - 1) * PW + pc);
                float4 ca, cb;
                coef(idprev, 0, ca, cb);
                const int kk = k - 1;
                const bool k1 = ST || kk >= 1, j1 = gj >= 1, i1a = gi >= 1;
                constexpr bool NOMASK = ST && PEC_TABLE;
                const float2 cex = NOMASK ? make_float2(ca.x, cb.x)
                                          : make_float2((j1 && k1) ? ca.x : 0.f, (j1 && k1) ? cb.x : 0.f);
                const float2 cey = NOMASK ? make_float2(ca.y, cb.y)
                                          : make_float2((i1a && k1) ? ca.y : 0.f, k1 ? cb.y : 0.f);
                const float2 cez = NOMASK ? make_float2(ca.z, cb.z)
                                          : make_float2((i1a && j1) ? ca.z : 0.f, j1 ? cb.z : 0.f);
                const float2 e2x = fma2(cex, sub2(sub2(h2z, hz_ym), sub2(h2y, h2py)), e1px);
                const float2 e2y = fma2(cey, sub2(sub2(h2x, h2px), sub2(h2z, make_float2(h2z_xm, h2z.x))), e1py);
                const float2 e2z = fma2(cez, sub2(sub2(h2y, make_float2(h2y_xm, h2y.x)), sub2(h2x, hx_ym)), e1pz);
                const long long g = (long long)kk * plane + (long long)gj * pitch + gi;
                if (out_a && ok && store_ok(P.status, g, 2, plane * nz)) {
                    Pair<T>::st_cs(dst0 + g, e2x.x, e2x.y);
                    Pair<T>::st_cs(dst0 + g + 1 * fstride, e2y.x, e2y.y);
                    Pair<T>::st_cs(dst0 + g + 2 * fstride, e2z.x, e2z.y);
                    Pair<T>::st_cs(dst0 + g + 3 * fstride, h2x.x, h2x.y);
                    Pair<T>::st_cs(dst0 + g + 4 * fstride, h2y.x, h2y.y);
                    Pair<T>::st_cs(dst0 + g + 5 * fstride, h2z.x, h2z.y);
                }
            }
            // ---------------- carry the z neighbours to the next plane
            h2px = h2x;
            h2py = h2y;
            h1px = h1x_;
            h1py = h1y_;
            h1pz = h1z_;
            e1px = e1x;
            e1py = e1y;
            e1pz = e1z;
            idprev = idpair;
            // ---------------- release unit k (and k+1 after the last plane)
            const bool last = !ST && k == kz1;
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
        };

        if (!SPLIT) {
#pragma unroll 2   // consecutive planes renamed instead of copied (the carried z neighbours)
            for (int k = kb; k <= kz1; ++k) plane_step(k, std::false_type{});
        } else {
            for (int k = kb; k <= kz1;) {
                if (k >= ks && k < kz1) {
#pragma unroll 2
                    for (; k < kz1; ++k) plane_step(k, std::true_type{});
                } else {
                    plane_step(k, std::false_type{});
                    ++k;
                }
            }
        }
    }
}

template <typename T, int TY, bool BATCH, int CM>
cudaError_t launch2_typed(const FusedLaunch &L, cudaStream_t s) {
    const int smem = smem2_bytes<T, TY>(L.stages);
    auto kern = fused2_step_kernel<T, TY, BATCH, CM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    Fused2Params P;
    P.recs = L.recs;
    P.step = L.step;
    P.launch_steps = L.launch_steps == 1 ? 1 : 2;
    P.ntiles = L.ntiles;
    P.parity = L.parity;
    P.status = L.status;
    P.stages = L.stages;
    P.slot_bytes = slot2_bytes<T, TY>();
    P.first = L.first;
    kern<<<L.grid, threads2<TY>(), smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T, int TY>
cudaError_t occupancy2_typed(int stages, int *n) {
    const int smem = smem2_bytes<T, TY>(stages);
    auto kern = fused2_step_kernel<T, TY, false, COEF_CLASS_ID_UNIFORM_H>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, threads2<TY>(), smem);
}

#define FDTD_DISPATCH2(storage, tile_y, ...)                                                          \
    do {                                                                                              \
        if (storage == 0) {                                                                           \
            if (tile_y == 8) { using T = float; constexpr int TY = 8; __VA_ARGS__; }                  \
            else if (tile_y == 12) { using T = float; constexpr int TY = 12; __VA_ARGS__; }           \
            else if (tile_y == 16) { using T = float; constexpr int TY = 16; __VA_ARGS__; }           \
        } else if (storage == 1) {                                                                    \
            if (tile_y == 8) { using T = __half; constexpr int TY = 8; __VA_ARGS__; }                 \
            else if (tile_y == 12) { using T = __half; constexpr int TY = 12; __VA_ARGS__; }          \
            else if (tile_y == 16) { using T = __half; constexpr int TY = 16; __VA_ARGS__; }          \
        } else if (storage == 2) {                                                                    \
            if (tile_y == 8) { using T = __nv_bfloat16; constexpr int TY = 8; __VA_ARGS__; }          \
            else if (tile_y == 12) { using T = __nv_bfloat16; constexpr int TY = 12; __VA_ARGS__; }   \
            else if (tile_y == 16) { using T = __nv_bfloat16; constexpr int TY = 16; __VA_ARGS__; }   \
        }                                                                                             \
    } while (0)

}  // namespace

int fused2_tile_w(int storage) { return storage == 0 ? Geom2<float>::W : Geom2<__half>::W; }

int fused2_smem_bytes(int storage, int tile_y, int stages) {
    int r = -1;
    FDTD_DISPATCH2(storage, tile_y, r = smem2_bytes<T, TY>(stages));
    return r;
}

cudaError_t fused2_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm) {
    cudaError_t e = cudaErrorInvalidValue;
    FDTD_DISPATCH2(storage, tile_y, e = occupancy2_typed<T, TY>(stages, ctas_per_sm));
    return e;
}

cudaError_t launch_fused2_step(int storage, const FusedLaunch &L, cudaStream_t s) {
    if (L.rows_per_warp == 2) return launch_fused2r_step(storage, L, s);
    if (L.ntiles <= 0) return cudaSuccess;
    if (L.stages < 3 || L.stages > 8) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    if (L.step || L.launch_steps == 1)   // a batch launch (or a one-step store launch)
        FDTD_DISPATCH2(storage, L.tile_y, e = (launch2_typed<T, TY, true, COEF_CLASS_ANY>(L, s)));
    else if (L.coef_class == COEF_CLASS_SCALAR)
        FDTD_DISPATCH2(storage, L.tile_y, e = (launch2_typed<T, TY, false, COEF_CLASS_SCALAR>(L, s)));
    else if (L.coef_class == COEF_CLASS_ID_UNIFORM_H)
        FDTD_DISPATCH2(storage, L.tile_y, e = (launch2_typed<T, TY, false, COEF_CLASS_ID_UNIFORM_H>(L, s)));
    else if (L.coef_class == COEF_CLASS_ID)
        FDTD_DISPATCH2(storage, L.tile_y, e = (launch2_typed<T, TY, false, COEF_CLASS_ID>(L, s)));
    else if (L.coef_class == COEF_CLASS_PEC_ID_UNIFORM_H)
        FDTD_DISPATCH2(storage, L.tile_y, e = (launch2_typed<T, TY, false, COEF_CLASS_PEC_ID_UNIFORM_H>(L, s)));
    else if (L.coef_class == COEF_CLASS_PEC_ID)
        FDTD_DISPATCH2(storage, L.tile_y, e = (launch2_typed<T, TY, false, COEF_CLASS_PEC_ID>(L, s)));
    else
        FDTD_DISPATCH2(storage, L.tile_y, e = (launch2_typed<T, TY, false, COEF_CLASS_ANY>(L, s)));
    return e;
}

}  // namespace fdtd
