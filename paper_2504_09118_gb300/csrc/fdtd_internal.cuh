// Internal definitions shared by the CUDA translation units of libfdtd.
//
// Device layout of one cavity (nx*ny*nz cells):
//   * Six "active" arrays, one per component, of nx*ny*nz entries (x pitch
//     padded to a multiple of 32 elements, rows 128-byte aligned), indexed by
//     the component's canonical (i,j,k) with i<nx, j<ny, k<nz.  Every entry the
//     leapfrog step can change lies in this range: at i = nx, j = ny or k = nz
//     E is tangential to a PEC face (always 0) and H is normal to it (constant).
//   * Two copies of the six arrays (ping-pong): a step reads copy s and writes
//     copy 1-s, so the fused kernel can recompute halo H from unmodified E.
//   * Three small FP32 "face" arrays holding the constant normal H on the far
//     faces (Hx at i = nx, Hy at j = ny, Hz at k = nz) for read-back and energy.
//   * Coefficients: scalars, or a one-byte material id per cell (active range)
//     indexing a table of (ce_x, ce_y, ce_z, ch_x, ch_y, ch_z), or six FP32 arrays.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

enum CoefMode : int { COEF_SCALAR = 0, COEF_ID8 = 1, COEF_FULL = 2 };

constexpr int kNumFields = 6;      // Ex, Ey, Ez, Hx, Hy, Hz
constexpr int kMaxTable = 256;
constexpr int kMaxPecMaterials = (kMaxTable - 1) / 8;   // 31: 1 + 8 x materials table entries
constexpr int kTileX = 64;         // fused kernel tile width along x (cells)
constexpr int kMapsPerCavity = 13; // [parity 0: 6 fields][parity 1: 6 fields][id]
constexpr int kMapSets = 4;        // box sets: one-step, two-step, fourth-order and three-step kernels

template <typename T> struct Storage;
template <> struct Storage<float> {
    static constexpr int kind = 0;
    static constexpr bool scaled = false;
    __device__ __forceinline__ static float load(float v) { return v; }
    __device__ __forceinline__ static float store(float v) { return v; }
};
template <> struct Storage<__half> {
    static constexpr int kind = 1;
    static constexpr bool scaled = true;
    __device__ __forceinline__ static float load(__half v) { return __half2float(v); }
    __device__ __forceinline__ static __half store(float v) { return __float2half_rn(v); }
};
template <> struct Storage<__nv_bfloat16> {
    static constexpr int kind = 2;
    static constexpr bool scaled = true;
    __device__ __forceinline__ static float load(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ __forceinline__ static __nv_bfloat16 store(float v) { return __float2bfloat16_rn(v); }
};

// Device-visible description of one cavity.
struct CavityDesc {
    int nx, ny, nz;
    int pitch;              // elements per row (x)
    long long plane;        // pitch * ny
    int coef_mode;          // CoefMode
    int ntab;               // table entries (COEF_ID8)
    int parity_off;         // current copy = launch parity ^ parity_off
    int pad0;
    float ce[3], ch[3];     // COEF_SCALAR
    float scale[6];         // storage scale s_c (1 for FP32)
    float inv_scale[6];
    void *buf[2][6];        // the two copies of the six active arrays
    const uint8_t *id;      // COEF_ID8: material id per active cell (same pitch)
    const float *table;     // COEF_ID8: ntab x 8 floats (ce xyz, pad, ch xyz, pad)
    const float *coef[6];   // COEF_FULL: ce x,y,z then ch x,y,z arrays (active range, same pitch)
    const CUtensorMap *maps;// fused kernel: kMapsPerCavity tensor maps (global memory)
    const float *face[3];   // constant normal H on the far faces: Hx[k][j] at i=nx, Hy[k][i] at j=ny, Hz[j][i] at k=nz
    const float *face_ch[3];// ch at those positions (NULL in COEF_SCALAR mode)
    const float *inv_table; // COEF_ID8: ntab x 8 floats of reciprocals (1/ce xyz, pad, 1/ch xyz, pad)
    float inv_ce[3], inv_ch[3];  // COEF_SCALAR reciprocals
    // Reductions sum over the cells of planes [kr_lo, kr_hi) (the owned cells of a z-slab; the whole
    // cavity otherwise) and include the far face k = nz when face_top is set.
    int kr_lo, kr_hi, face_top, pad1;
};

// Physical (unscaled) value of field f at linear offset off of copy `copy`.
template <typename T>
__device__ __forceinline__ float ld_field(const CavityDesc &d, int copy, int f, long long off) {
    const T v = static_cast<const T *>(d.buf[copy][f])[off];
    float x = Storage<T>::load(v);
    if (Storage<T>::scaled) x *= d.inv_scale[f];
    return x;
}

template <typename T>
__device__ __forceinline__ void st_field(const CavityDesc &d, int copy, int f, long long off, float x) {
    if (Storage<T>::scaled) x *= d.scale[f];
    static_cast<T *>(d.buf[copy][f])[off] = Storage<T>::store(x);
}

// 1/ce (c = 0..2) or 1/ch (c = 3..5) of the cell at active offset off.
__device__ __forceinline__ float ld_inv_coef(const CavityDesc &d, int c, long long off) {
    if (d.coef_mode == COEF_SCALAR) return c < 3 ? d.inv_ce[c] : d.inv_ch[c - 3];
    if (d.coef_mode == COEF_ID8) return d.inv_table[8 * d.id[off] + (c < 3 ? c : c + 1)];
    return 1.0f / d.coef[c][off];
}

// ce (c = 0..2) or ch (c = 3..5) of the cell at active offset off.
__device__ __forceinline__ float ld_coef(const CavityDesc &d, int c, long long off) {
    if (d.coef_mode == COEF_SCALAR) return c < 3 ? d.ce[c] : d.ch[c - 3];
    if (d.coef_mode == COEF_ID8) return d.table[8 * d.id[off] + (c < 3 ? c : c + 1)];
    return d.coef[c][off];
}

// One unit of fused-kernel work: a TX x TY column of cells over planes [kz0, kz1).
struct TileDesc {
    int cav;
    int x0, y0;
    int kz0, kz1;
    int pad[3];
};

// Everything the fused kernel needs about one tile, built on the host (256 bytes,
// copied by the kernel's producer warp into shared memory when the tile starts).
struct alignas(16) TileRec {
    int x0, y0, kz0, kz1;
    int nx, ny, pitch, mode;     // mode: CoefMode (COEF_SCALAR or COEF_ID8)
    long long plane;             // pitch * ny
    int ch_uniform;              // ch is the same in every cell (scalars in ch[])
    int parity_off;              // source copy = launch parity ^ parity_off
    // Coefficients in storage units: with E stored as s_E*E and H as s_H*H, ce*s_E/s_H and
    // ch*s_H/s_E (both 1 for FP32 storage), so the kernel never rescales a field value.
    float ce[3], ch[3];          // scalar coefficients (COEF_SCALAR; ch also when ch_uniform)
    const float4 *table;         // COEF_ID8: per id two float4: (ce x,y,z,0), (ch x,y,z,0), folded
    const CUtensorMap *maps;     // kMapsPerCavity tensor maps in global memory
    void *dst[2][6];             // both copies of the six active arrays
    long long stop;              // batch step clock at which this tile's member has taken all its steps
    int ntab;                    // COEF_ID8: table entries
    int nz;
    int id_x0;                   // two-step kernel: x origin of the id box (a multiple of 16)
    int pad[13];
};
static_assert(sizeof(TileRec) == 256, "TileRec must be 256 bytes");

// Status bits latched by kernels into the device status word.
enum : int { STATUS_TIMEOUT = 1, STATUS_BADINDEX = 2 };

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Suspend-time hint (ns) of one mbarrier poll; 0 polls without a hint.
#ifndef FDTD_WAIT_HINT_NS
#define FDTD_WAIT_HINT_NS 0
#endif

// One poll of the phase with the given parity; may sleep in hardware up to the hint.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
#if FDTD_WAIT_HINT_NS > 0
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"((uint32_t)FDTD_WAIT_HINT_NS)
        : "memory");
#else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
#endif
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `bar` with the given parity to complete, for at most
// limit_ns nanoseconds of wall time.  Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        for (int r = 0; r < 4; ++r)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// Bounded wait that also gives up when another warp of the CTA has raised *abort; a wait that
// runs out raises it.  sleep_ns > 0 sleeps between polls (for waits off the critical path).
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                                    volatile int *abort, unsigned sleep_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (sleep_ns) __nanosleep(sleep_ns);
        for (int r = 0; r < 4; ++r)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (global_timer_ns() - t0 > limit_ns) {
            *abort = 1;
            return false;
        }
    }
}

// As mbar_wait_bounded, but sleeps sleep_ns between polls (for a thread whose wait is not on the
// critical path, so that it does not take issue slots from the warps doing the arithmetic).
__device__ __forceinline__ bool mbar_wait_bounded_sleep(uint64_t *bar, uint32_t parity, uint64_t limit_ns,
                                                        unsigned sleep_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        __nanosleep(sleep_ns);
        if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbarrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
// 4-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_4d(void *smem_dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::
            "r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *smem_dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace fdtd
