// Host-side launchers of libfdtd's kernels (C++ linkage, internal to the library).
#pragma once

#include "fdtd_internal.cuh"

namespace fdtd {

// Canonical FP32 component -> active array (scaled, rounded to storage), tangential E zeroed,
// far-face normal H -> face array (FP32, after the same rounding).
cudaError_t launch_pack(int storage, const CavityDesc &d, int copy, int comp, const float *canon, float *face,
                        cudaStream_t s);
// Active array (+ face) -> canonical FP32 component, zero outside the extent.
cudaError_t launch_unpack(int storage, const CavityDesc &d, int copy, int comp, float *canon, cudaStream_t s);
// max |canon| over the component's extent, as float bits atomically max-ed into *out (must start at 0).
cudaError_t launch_maxabs(const float *canon, int comp, int nx, int ny, int nz, unsigned *out, cudaStream_t s);
// One unfused step in place on copy `copy`: H kernel then E kernel.
cudaError_t launch_simple_step(int storage, const CavityDesc &d, int copy, cudaStream_t s);
// Reductions accumulated in FP64: what == 0 gives out[0] = sum E^2/ce + H.(H - ch curl E)/ch;
// what == 1 gives out[1] = sum divE^2, out[2] = sum divH^2.  partial holds nblocks*3 doubles.
// order 4 takes the curl and divergences of the fourth-order scheme.
cudaError_t launch_reductions(int storage, const CavityDesc &d, int copy, int what, double *partial, int nblocks,
                              double *out, cudaStream_t s, int order = 2);
// Fourth-order scheme (k_order4.cu): one unfused step in place on copy `copy`, and the per-block
// partials of its reductions (same layout as launch_reductions' partial).
cudaError_t launch_simple4_step(int storage, const CavityDesc &d, int copy, cudaStream_t s);
cudaError_t launch_reductions4(int storage, const CavityDesc &d, int copy, int what, double *partial, int nblocks,
                               cudaStream_t s);
int reduction_blocks();

struct FusedLaunch {
    const TileRec *recs;       // device array, one record per tile
    const long long *step;     // device step clock compared with TileRec::stop (NULL: no tile skipped)
    int ntiles;
    int parity;
    int *status;
    int tile_y;
    int stages;
    int grid;
    int inject_timeout_us;     // >0: do not issue the CTA 0's first unit; wait limit in us
    const int *first;          // device, grid + 1 entries: CTA b takes tiles [first[b], first[b+1]) in order
                               // (NULL: CTA b takes tiles b, b + grid, b + 2 grid, ...)
    int launch_steps;          // two-step kernel: 2, or 1 (every tile stores its level-1 result only)
    int rows_per_warp;         // two-step kernel: 1 (k_fused2.cu) or 2 (k_fused2r.cu); 0 means 1
    int coef_class;            // CoefClass shared by every tile (COEF_CLASS_ANY: read from each record)
};
// Coefficient layout shared by all tiles of a launch, so that a kernel can be compiled for it.
enum CoefClass : int {
    COEF_CLASS_ANY = 0,        // tiles may differ (batches of mixed members): the record's mode decides
    COEF_CLASS_SCALAR = 1,     // COEF_SCALAR: three ce and three ch for the whole cavity
    COEF_CLASS_ID_UNIFORM_H = 2,  // COEF_ID8 with the same ch in every cell
    COEF_CLASS_ID = 3,         // COEF_ID8 with ce and ch per material id
    // COEF_ID8 whose ids and table code the PEC faces (fdtd_ctx::id_pec): no per-cell masks in the kernel
    COEF_CLASS_PEC_ID_UNIFORM_H = 4,
    COEF_CLASS_PEC_ID = 5,
};
inline int coef_class_of(int coef_mode, int ch_uniform, bool pec_ids) {
    if (coef_mode == COEF_SCALAR) return COEF_CLASS_SCALAR;
    if (coef_mode == COEF_ID8) {
        if (pec_ids) return ch_uniform ? COEF_CLASS_PEC_ID_UNIFORM_H : COEF_CLASS_PEC_ID;
        return ch_uniform ? COEF_CLASS_ID_UNIFORM_H : COEF_CLASS_ID;
    }
    return COEF_CLASS_ANY;
}
// Shared memory bytes and max co-resident CTAs per SM for a fused configuration.
int fused_smem_bytes(int storage, int tile_y, int stages);
cudaError_t fused_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm);
cudaError_t launch_fused_step(int storage, const FusedLaunch &L, cudaStream_t s);
// *counter += 1 on the stream (advances a batch's device launch counter after each step).
// Point currents and probes applied after a step (k_extras.cu).
struct ExtrasParams {
    long long *clock;          // device: steps taken since fdtd_set_fields; advanced by the launch
    int nsrc, wave_len;
    const int *src_comp;       // 0..2 (Ex, Ey, Ez)
    const long long *src_off;  // active-array offsets
    const float *wave;         // nsrc x wave_len: J^{n+1/2} of step n
    float dx;
    int nprobe, capacity;
    long long probe_start;     // step index of the probe buffer's first sample
    const int *probe_comp;     // 0..5
    const long long *probe_off;
    float *probe_buf;          // nprobe x capacity, physical units
};
cudaError_t launch_extras(int storage, const CavityDesc &d, int copy, const ExtrasParams &X, cudaStream_t s);

// Adds inc to the device step clock of a batch (one thread; ordered after the launch it follows).
cudaError_t launch_step_counter(long long *counter, int inc, cudaStream_t s);
// Two-step (temporal blocking) kernel: output tile width along x, shared memory, occupancy, launch.
int fused2_tile_w(int storage);
int fused2_smem_bytes(int storage, int tile_y, int stages);
cudaError_t fused2_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm);
cudaError_t launch_fused2_step(int storage, const FusedLaunch &L, cudaStream_t s);
// The two-step kernel with two rows per consumer warp (k_fused2r.cu; tile heights 12 and 16): the same
// tiles, boxes and results, a different split of the rows over the warps.
int fused2r_smem_bytes(int storage, int tile_y, int stages);
cudaError_t fused2r_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm);
cudaError_t launch_fused2r_step(int storage, const FusedLaunch &L, cudaStream_t s);
// Three-step (T = 3) kernel (k_fused3.cu; single cavities, tile heights 8, 10 and 12): output tile width along x,
// shared memory, occupancy, launch.
int fused3_tile_w();
int fused3_smem_bytes(int storage, int tile_y, int stages);
cudaError_t fused3_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm);
cudaError_t launch_fused3_step(int storage, const FusedLaunch &L, cudaStream_t s);
// Fused fourth-order kernel (k_fused4.cu): shared memory, occupancy, launch (stages 4..8).
int fused4_smem_bytes(int storage, int tile_y, int stages);
cudaError_t fused4_occupancy(int storage, int tile_y, int stages, int *ctas_per_sm);
cudaError_t launch_fused4_step(int storage, const FusedLaunch &L, cudaStream_t s);
// Box sizes used to encode the tensor maps of the fused kernel.
void fused_box(int storage, int tile_y, int *box_x, int *box_y, int *halo_x);

}  // namespace fdtd
