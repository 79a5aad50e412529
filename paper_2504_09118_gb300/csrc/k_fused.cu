// Fused Yee step (H then E in one pass over HBM) for sm_103a.
//
// The update is Eq. 2 of the paper in the order of Listing 1: H^{n+1/2} from
// curl E^n, then E^{n+1} from curl H^{n+1/2}, PEC by index predicates (tangential
// E is never updated; normal H on a face sees a zero curl).  Reads copy s of
// the six fields and writes copy 1-s (ping-pong), so a tile can recompute the
// H values on its lower x/y halo from unmodified E instead of waiting for the
// neighbouring tile.
//
// Work decomposition: a tile is a 64 x TY column of cells over planes
// [kz0, kz1).  Persistent CTAs take tiles round-robin (tile = blockIdx.x +
// m * gridDim.x) and march each tile upward in z.  Plane k needs "unit" k (all
// six fields and the material id at plane k, with a halo of one cell in x and
// y, padded in x to the 16-byte TMA granule) and unit k+1 (E at k+1 for the z
// derivative of the H update).  One thread streams units into an S-slot shared
// memory ring with 3-D TMA loads completing on per-slot mbarriers; the stream
// runs on across tile boundaries so the pipeline never drains between tiles.
// H^{n+1/2}(k-1) at the thread's own cells stays in registers for the
// z-derivative of the E update; a tile starting at kz0 > 0 first recomputes
// plane kz0-1 (a "prologue" plane).
//
// Per plane and cell, HBM sees 6 loads and 6 stores of the storage type plus
// one material-id byte (24+24+1 = 49 B/cell in FP32); halo rows are re-read
// from L2.  Every mbarrier wait is bounded in wall time (globaltimer); on
// expiry the CTA latches STATUS_TIMEOUT, drains its in-flight copies (bounded
// again) and exits.
#include "launch.h"

namespace fdtd {

namespace {

constexpr int TX = kTileX;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: far beyond any healthy TMA latency

template <typename T> struct FusedGeom {
    static constexpr int HX = 16 / (int)sizeof(T);     // x halo rounded to a 16-byte TMA granule
    static constexpr int BX = TX + 2 * HX;             // field box width (elements)
    static constexpr int IDX_HALO = 16;                // id box starts 16 bytes left of x0
    static constexpr int IBX = TX + IDX_HALO;          // id box width (bytes)
};

struct FusedParams {
    const CavityDesc *cav;
    const TileDesc *tiles;
    int ntiles;
    int parity;
    int *status;
    int stages;
    int slot_bytes;
    int inject_timeout_us;
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
// Each TMA destination box starts on a 128-byte boundary.
template <typename T, int TY>
__host__ __device__ constexpr int field_box_stride() {
    return align_up(field_box_bytes<T, TY>(), 128);
}
template <typename T, int TY>
__host__ __device__ constexpr int slot_bytes() {
    return align_up(6 * field_box_stride<T, TY>() + id_box_bytes<TY>(), 128);
}
template <int TY>
__host__ __device__ constexpr int hplane_floats() {
    return 3 * (TY + 1) * (TX + 1);
}
template <typename T, int TY>
__host__ __device__ constexpr int smem_bytes(int stages) {
    return 128 /*barriers*/ + kMaxTable * 8 * 4 /*table*/ + align_up(hplane_floats<TY>() * 4, 128) +
           stages * slot_bytes<T, TY>() + 128 /*alignment slack*/;
}

// Producer-side view of one tile (kept in registers by the issuing thread).
struct ProdTile {
    const CUtensorMap *maps;
    int src;
    int has_id;
    int x0, y0, k, kend;   // next plane to issue, last plane (inclusive)
};

template <typename T, int TY>
__device__ __forceinline__ void load_prod_tile(const FusedParams &P, int t, ProdTile &pt) {
    const TileDesc td = P.tiles[t];
    const CavityDesc &cd = P.cav[td.cav];
    pt.maps = cd.maps;
    pt.src = P.parity ^ cd.parity_off;
    pt.has_id = cd.coef_mode == COEF_ID8;
    pt.x0 = td.x0;
    pt.y0 = td.y0;
    pt.k = td.kz0 > 0 ? td.kz0 - 1 : td.kz0;
    pt.kend = td.kz1;
}

template <typename T, int TY, int NT>
__global__ void __launch_bounds__(NT) fused_step_kernel(const FusedParams P) {
    using G = FusedGeom<T>;
    constexpr int HX = G::HX, BX = G::BX, BY = TY + 2, HP = TX + 1;
    constexpr int FB = field_box_bytes<T, TY>();      // bytes the TMA writes per field box
    constexpr int FS = field_box_stride<T, TY>();     // byte stride between boxes in a slot
    constexpr int FE = FS / (int)sizeof(T);           // element stride between boxes
    constexpr int R = TX * TY / NT;                   // interior cells per thread per plane
    static_assert(TX * TY % NT == 0, "tile must split evenly over the block");

    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    float *tab = reinterpret_cast<float *>(smem + 128);
    float *hn = tab + kMaxTable * 8;
    unsigned char *slots = reinterpret_cast<unsigned char *>(hn) + align_up(hplane_floats<TY>() * 4, 128);

    const int tid = threadIdx.x;
    const int S = P.stages;
    const int SB = P.slot_bytes;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_mbarrier_init();
        fence_proxy_async_smem();
    }
    __syncthreads();

    // ---------------- producer state (thread 0 only)
    int p_t = blockIdx.x;
    int issued = 0, released = 0;
    ProdTile pt{};
    const bool inject = P.inject_timeout_us > 0 && blockIdx.x == 0;
    const uint64_t wait_limit = inject ? (uint64_t)P.inject_timeout_us * 1000ull : kWaitLimitNs;

    auto issue_more = [&]() {
        while (issued - released < S && p_t < P.ntiles) {
            const int slot = issued % S;
            unsigned char *dst = slots + slot * SB;
            uint64_t *bar = &full[slot];
            if (inject && issued == 0) {
                // fault injection: leave slot 0's barrier un-armed so its wait runs out
            } else {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, 6 * FB + (pt.has_id ? id_box_bytes<TY>() : 0));
                const CUtensorMap *m = pt.maps + pt.src * 6;
#pragma unroll
                for (int f = 0; f < 6; ++f) tma_load_3d(dst + f * FS, m + f, pt.x0 - HX, pt.y0 - 1, pt.k, bar);
                if (pt.has_id)
                    tma_load_3d(dst + 6 * FS, pt.maps + 12, pt.x0 - G::IDX_HALO, pt.y0 - 1, pt.k, bar);
            }
            ++issued;
            if (++pt.k > pt.kend) {
                p_t += gridDim.x;
                if (p_t < P.ntiles) load_prod_tile<T, TY>(P, p_t, pt);
            }
        }
    };
    if (tid == 0 && p_t < P.ntiles) {
        load_prod_tile<T, TY>(P, p_t, pt);
        issue_more();
    }

    // ---------------- consumers (all threads, thread 0 included)
    int u_base = 0;
    int loaded_tab_cav = -1;
    float hprev_x[R], hprev_y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) hprev_x[r] = hprev_y[r] = 0.f;

    for (int t = blockIdx.x; t < P.ntiles; t += gridDim.x) {
        const TileDesc td = P.tiles[t];
        const CavityDesc &cd = P.cav[td.cav];
        const int nx = cd.nx, ny = cd.ny;
        const int pitch = cd.pitch;
        const long long plane = cd.plane;
        const int mode = cd.coef_mode;
        const int dstc = (P.parity ^ cd.parity_off) ^ 1;
        float inv_s[6], sc[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            inv_s[f] = cd.inv_scale[f];
            sc[f] = cd.scale[f];
        }
        T *dstp[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) dstp[f] = static_cast<T *>(cd.buf[dstc][f]);
        float ce_s[3], ch_s[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ce_s[c] = cd.ce[c];
            ch_s[c] = cd.ch[c];
        }
        if (mode == COEF_ID8 && loaded_tab_cav != td.cav) {
            for (int e = tid; e < cd.ntab * 8; e += NT) tab[e] = cd.table[e];
            loaded_tab_cav = td.cav;   // made visible by the barrier at the top of the first iteration
        }
        const int kb = td.kz0 > 0 ? td.kz0 - 1 : td.kz0;

        for (int k = kb; k < td.kz1; ++k) {
            const int ua = u_base + (k - kb), ub = ua + 1;
            bool ok = mbar_wait_bounded(&full[ua % S], (ua / S) & 1, wait_limit);
            ok = ok && mbar_wait_bounded(&full[ub % S], (ub / S) & 1, wait_limit);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(P.status, STATUS_TIMEOUT);
                    // drain this CTA's copies still in flight (bounded again) before shared memory goes away
                    for (int u = released; u < issued; ++u) {
                        if (inject && u == 0) continue;
                        mbar_wait_bounded(&full[u % S], (u / S) & 1, kWaitLimitNs);
                    }
                }
                __syncthreads();
                return;
            }
            const unsigned char *sa = slots + (ua % S) * SB;
            const unsigned char *sbb = slots + (ub % S) * SB;
            const T *Ea = reinterpret_cast<const T *>(sa);             // fields 0..5 of plane k
            const T *Eb = reinterpret_cast<const T *>(sbb);            // fields 0..2 of plane k+1
            const uint8_t *ida = sa + 6 * FS;
            const bool prologue = k < td.kz0;
            const long long zoff = (long long)k * plane;

            auto F = [&](const T *base, int f, int bx, int by) -> float {
                float v = Storage<T>::load(base[f * FE + by * BX + bx]);
                if (Storage<T>::scaled) v *= inv_s[f];
                return v;
            };
            auto coef = [&](int x, int y, int c) -> float {   // c: 0..2 ce, 3..5 ch
                if (mode == COEF_ID8) {
                    const int id = ida[(y + 1) * G::IBX + (x + G::IDX_HALO)];
                    return tab[id * 8 + (c < 3 ? c : c + 1)];
                }
                return c < 3 ? ce_s[c] : ch_s[c - 3];
            };
            // H^{n+1/2} at local (x, y) of plane k, from unit k (E, H) and unit k+1 (E).
            auto h_update = [&](int x, int y, float &hx, float &hy, float &hz) {
                const int bx = x + HX, by = y + 1;
                const float ex = F(Ea, 0, bx, by), ey = F(Ea, 1, bx, by), ez = F(Ea, 2, bx, by);
                const float ex_y1 = F(Ea, 0, bx, by + 1), ez_y1 = F(Ea, 2, bx, by + 1);
                const float ey_x1 = F(Ea, 1, bx + 1, by), ez_x1 = F(Ea, 2, bx + 1, by);
                const float ex_z1 = F(Eb, 0, bx, by), ey_z1 = F(Eb, 1, bx, by);
                hx = F(Ea, 3, bx, by) - coef(x, y, 3) * ((ez_y1 - ez) - (ey_z1 - ey));
                hy = F(Ea, 4, bx, by) - coef(x, y, 4) * ((ex_z1 - ex) - (ez_x1 - ez));
                hz = F(Ea, 5, bx, by) - coef(x, y, 5) * ((ey_x1 - ey) - (ex_y1 - ex));
            };

            // ---- phase A: H on the interior (kept in registers and shared memory, stored) and the lower halo
            float hxi[R], hyi[R], hzi[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int p = tid + r * NT;
                const int x = p % TX, y = p / TX;
                h_update(x, y, hxi[r], hyi[r], hzi[r]);
            }
            if (!prologue) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int p = tid + r * NT;
                    const int x = p % TX, y = p / TX;
                    const int o = (y + 1) * HP + (x + 1);
                    hn[o] = hxi[r];
                    hn[(TY + 1) * HP + o] = hyi[r];
                    hn[2 * (TY + 1) * HP + o] = hzi[r];
                    const int gi = td.x0 + x, gj = td.y0 + y;
                    if (gi < nx && gj < ny) {
                        const long long go = zoff + (long long)gj * pitch + gi;
                        dstp[3][go] = Storage<T>::store(Storage<T>::scaled ? hxi[r] * sc[3] : hxi[r]);
                        dstp[4][go] = Storage<T>::store(Storage<T>::scaled ? hyi[r] * sc[4] : hyi[r]);
                        dstp[5][go] = Storage<T>::store(Storage<T>::scaled ? hzi[r] * sc[5] : hzi[r]);
                    }
                }
                // halo: row y = -1 (Hx, Hz used by Ex/Ez) and column x = -1 (Hy, Hz used by Ey/Ez)
                for (int h = tid; h < TX + TY; h += NT) {
                    const int x = h < TX ? h : -1;
                    const int y = h < TX ? -1 : h - TX;
                    float a, b, c;
                    h_update(x, y, a, b, c);
                    const int o = (y + 1) * HP + (x + 1);
                    hn[o] = a;
                    hn[(TY + 1) * HP + o] = b;
                    hn[2 * (TY + 1) * HP + o] = c;
                }
            }
            __syncthreads();

            // ---- phase B: E^{n+1} on the interior
            if (!prologue) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int p = tid + r * NT;
                    const int x = p % TX, y = p / TX;
                    const int gi = td.x0 + x, gj = td.y0 + y;
                    const int o = (y + 1) * HP + (x + 1);
                    const float hx = hxi[r], hy = hyi[r], hz = hzi[r];
                    const float hx_ym = hn[o - HP];
                    const float hz_ym = hn[2 * (TY + 1) * HP + o - HP];
                    const float hy_xm = hn[(TY + 1) * HP + o - 1];
                    const float hz_xm = hn[2 * (TY + 1) * HP + o - 1];
                    const int bx = x + HX, by = y + 1;
                    float ex = F(Ea, 0, bx, by), ey = F(Ea, 1, bx, by), ez = F(Ea, 2, bx, by);
                    if (gj >= 1 && k >= 1) ex += coef(x, y, 0) * ((hz - hz_ym) - (hy - hprev_y[r]));
                    if (gi >= 1 && k >= 1) ey += coef(x, y, 1) * ((hx - hprev_x[r]) - (hz - hz_xm));
                    if (gi >= 1 && gj >= 1) ez += coef(x, y, 2) * ((hy - hy_xm) - (hx - hx_ym));
                    if (gi < nx && gj < ny) {
                        const long long go = zoff + (long long)gj * pitch + gi;
                        dstp[0][go] = Storage<T>::store(Storage<T>::scaled ? ex * sc[0] : ex);
                        dstp[1][go] = Storage<T>::store(Storage<T>::scaled ? ey * sc[1] : ey);
                        dstp[2][go] = Storage<T>::store(Storage<T>::scaled ? ez * sc[2] : ez);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                hprev_x[r] = hxi[r];
                hprev_y[r] = hyi[r];
            }
            __syncthreads();
            if (tid == 0) {
                released += (k == td.kz1 - 1) ? 2 : 1;
                issue_more();
            }
        }
        u_base += td.kz1 - kb + 1;
    }
}

template <typename T, int TY>
constexpr int threads_for() {
    return TX * TY / 2;
}

template <typename T, int TY>
cudaError_t launch_typed(const FusedLaunch &L, cudaStream_t s) {
    constexpr int NT = threads_for<T, TY>();
    const int smem = smem_bytes<T, TY>(L.stages);
    auto kern = fused_step_kernel<T, TY, NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    FusedParams P;
    P.cav = L.cav;
    P.tiles = L.tiles;
    P.ntiles = L.ntiles;
    P.parity = L.parity;
    P.status = L.status;
    P.stages = L.stages;
    P.slot_bytes = slot_bytes<T, TY>();
    P.inject_timeout_us = L.inject_timeout_us;
    kern<<<L.grid, NT, smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T, int TY>
cudaError_t occupancy_typed(int stages, int *n) {
    constexpr int NT = threads_for<T, TY>();
    const int smem = smem_bytes<T, TY>(stages);
    auto kern = fused_step_kernel<T, TY, NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, NT, smem);
}

#define FDTD_DISPATCH(storage, tile_y, ...)                                                         \
    do {                                                                                             \
        if (storage == 0) {                                                                          \
            if (tile_y == 4) { using T = float; constexpr int TY = 4; __VA_ARGS__; }                        \
            else if (tile_y == 8) { using T = float; constexpr int TY = 8; __VA_ARGS__; }                   \
            else if (tile_y == 16) { using T = float; constexpr int TY = 16; __VA_ARGS__; }                 \
        } else if (storage == 1) {                                                                   \
            if (tile_y == 4) { using T = __half; constexpr int TY = 4; __VA_ARGS__; }                       \
            else if (tile_y == 8) { using T = __half; constexpr int TY = 8; __VA_ARGS__; }                  \
            else if (tile_y == 16) { using T = __half; constexpr int TY = 16; __VA_ARGS__; }                \
        } else if (storage == 2) {                                                                   \
            if (tile_y == 4) { using T = __nv_bfloat16; constexpr int TY = 4; __VA_ARGS__; }                \
            else if (tile_y == 8) { using T = __nv_bfloat16; constexpr int TY = 8; __VA_ARGS__; }           \
            else if (tile_y == 16) { using T = __nv_bfloat16; constexpr int TY = 16; __VA_ARGS__; }         \
        }                                                                                            \
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
    cudaError_t e = cudaErrorInvalidValue;
    FDTD_DISPATCH(storage, L.tile_y, e = launch_typed<T, TY>(L, s));
    return e;
}

void fused_box(int storage, int tile_y, int *box_x, int *box_y, int *halo_x) {
    const int esz = storage == 0 ? 4 : 2;
    *halo_x = 16 / esz;
    *box_x = TX + 2 * (16 / esz);
    *box_y = tile_y + 2;
}

}  // namespace fdtd
