// Internal definitions shared by the host-side translation units of libfdtd (the C ABI of
// include/fdtd.h): the context and batch objects, the stream-ordered device pool, the launch
// planner and the helpers the entry points share.  Not part of the ABI.
#pragma once

#include <cudaTypedefs.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <queue>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/fdtd.h"
#include "launch.h"

namespace fdtd {

namespace {
// NVTX range over a library call (visible in Nsight Systems / Compute timelines; header-only NVTX3,
// a no-op unless a tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

struct GraphKey {
    int steps, parity, kind = 0;
    bool operator<(const GraphKey &o) const {
        if (kind != o.kind) return kind < o.kind;
        return steps != o.steps ? steps < o.steps : parity < o.parity;
    }
};


}  // namespace fdtd

// The C ABI's opaque handles are global-namespace types; their members use the library's types.
using namespace fdtd;

struct fdtd_ctx {
    int nx = 0, ny = 0, nz = 0;
    double dt = 0, dx = 0;
    int storage = 0;
    cudaStream_t stream = nullptr;
    int pitch = 0;
    size_t arr_elems = 0;
    void *fields[2][6] = {};
    float *face[3] = {}, *face_ch[3] = {};
    int coef_mode = COEF_SCALAR;
    float ce_s[3] = {}, ch_s[3] = {};
    uint8_t *id = nullptr;
    float *table = nullptr, *inv_table = nullptr;
    float *table_fused = nullptr;     // table with the storage-scale ratios folded in (fused kernel)
    std::vector<float> host_table;    // 8 floats per entry: ce xyz, pad, ch xyz, pad
    int ntab = 0;
    // PEC as materials (two-step kernel, up to kMaxPecMaterials materials): per cell 1 + id + ntab faces
    // (bit 0: i = 0, bit 1: j = 0, bit 2: k = 0), 0 outside the cavity; table_pec holds the folded
    // coefficients with the E components tangential to those faces set to zero (entry 0: ce = 0)
    uint8_t *id_pec = nullptr;
    float *table_pec = nullptr;
    int ntab_pec = 0;
    float *coef_full[6] = {};
    float scale[6] = {1, 1, 1, 1, 1, 1};
    int cur = 0;
    long long steps = 0;
    bool has_fields = false;
    int *d_status = nullptr;
    double *d_partial = nullptr, *d_out = nullptr;
    float *d_stage = nullptr;    // canonical staging buffer for host transfers (lazy)
    float *d_stage2 = nullptr;   // second staging buffer: host loads copy one field while packing another
    cudaStream_t copy_stream = nullptr;   // host-to-device copies of fdtd_set_fields (lazy)
    cudaEvent_t staged[2] = {nullptr, nullptr}, packed[2] = {nullptr, nullptr};
    // fdtd_prefetch_fields: six canonical arrays copied from the host on the copy stream while the
    // context computes; fdtd_set_fields_prefetched loads them (lazy)
    float *d_prefetch = nullptr;
    cudaEvent_t prefetched = nullptr, prefetch_free = nullptr;
    bool prefetch_pending = false;
    unsigned *d_max = nullptr;
    CUtensorMap *d_maps = nullptr;          // kMapSets x kMapsPerCavity
    std::vector<CUtensorMap> host_maps[kMapSets];
    int maps_by[kMapSets] = {0, 0, 0, 0};   // box height each map set was encoded for (0: not yet)
    CavityDesc *d_desc = nullptr;
    struct TileList {
        TileRec *d = nullptr;   // records, followed by the per-CTA range offsets
        int *first = nullptr;   // inside the same allocation as d
        int n = 0, grid = 0, key = 0;
    } tl[4];                                // [0] one-step, [1] two-step, [2] fourth-order, [3] three-step kernel
    int order = 2;                          // spatial order of the differences (2: Eq. 2, 4: the (2,4) scheme)
    double courant = 0.0;                   // max over cells of 3 ce ch (stable for order 2 when <= 1)
    int ch_uniform = 1;
    fdtd_tuning tuning{};
    std::map<fdtd::GraphKey, cudaGraphExec_t> graphs;
    int inject_us = 0;
    // point currents and probes (fdtd_set_sources / fdtd_set_probes): run after every step
    int nsrc = 0, wave_len = 0, nprobe = 0, probe_cap = 0;
    long long probe_start = 0;         // step index of a probe buffer's first sample
    int *d_src_comp = nullptr, *d_probe_comp = nullptr;
    long long *d_src_off = nullptr, *d_probe_off = nullptr;
    float *d_wave = nullptr, *d_probe_buf = nullptr;
    long long *d_xclock = nullptr;     // device: steps taken since fdtd_set_fields (advanced by the extras launch)
    long long bytes = 0;
    fdtd_batch *batch = nullptr;
    float fixed_scale[2] = {0.f, 0.f};      // fdtd_set_storage_scales: s_E, s_H of later loads (0: from the data)
    // z-slab of a larger cavity (fdtd_create_slab): local planes 0..nz are global planes z_off..z_off + nz;
    // g_lo / g_hi ghost cells lie below / above the owned cells (0 on a side that is a real PEC wall);
    // left[side] is how many more steps the owned cells stay exact before that side needs an import
    struct SlabInfo {
        int on = 0, nz_global = 0, z_off = 0, g_lo = 0, g_hi = 0, ghost = 0;
        int left[2] = {0, 0};
        cudaEvent_t ev = nullptr;
    } slab;
    std::string err;
};

struct fdtd_batch {
    struct Member {
        fdtd_ctx *c;
        int cur0;               // member's current copy when it joined
        long long join;         // batch step clock at which it joined
        long long join_launch;  // batch launch count at which it joined
        long long stop;         // step clock at which it has taken all its steps (LLONG_MAX: no limit)
        long long steps0;       // its step count when it joined
        long long nlaunch;      // launches it took part in since joining (each flips its copy)
    };
    int storage = 0;
    int order = 2;                   // spatial order of every member (set by the first member joining)
    cudaStream_t stream = nullptr;
    std::vector<Member> members;
    long long step = 0;              // step clock: steps enqueued so far (a two-step launch advances it by 2)
    long long launches = 0;          // launches enqueued so far; the next launch has parity launches & 1
    long long *d_step = nullptr;     // device copy of the step clock (advanced by a kernel after each launch)
    fdtd_tuning tuning{};
    TileRec *d_tiles = nullptr;      // tile records, then (at d_first) the per-CTA range offsets
    int *d_first = nullptr;          // grid + 1 offsets when the tiles are assigned to CTAs on the host, else NULL
    int tiles_cap = 0, ntiles = 0, grid = 0;
    // pinned staging of the tile-list uploads, two buffers used in turn: a copy from pageable memory may
    // wait for the stream, which would drain the queued launches at every change of membership
    void *h_stage[2] = {nullptr, nullptr};
    size_t h_stage_cap[2] = {0, 0};
    cudaEvent_t h_stage_ev[2] = {nullptr, nullptr};   // recorded after each buffer's last upload
    int h_stage_next = 0;
    bool dirty = true;
    int *d_status = nullptr;
    cudaEvent_t done_ev = nullptr;   // recorded at member removal; the member's stream waits on it
    // Completion marks: after each fdtd_batch_step call, an event and the clock it brings the batch
    // to.  A removed member's stream waits only for the first mark at or past the clock at which the
    // member took its last step (later launches skip it), not for everything enqueued since.
    std::deque<std::pair<long long, cudaEvent_t>> marks;
    std::vector<cudaEvent_t> free_marks;
    std::map<fdtd::GraphKey, cudaGraphExec_t> graphs;
    // (batch clock when retired, graph): destroyed once a completion mark at or past that clock has passed,
    // or at the next synchronisation point
    std::vector<std::pair<long long, cudaGraphExec_t>> retired_graphs;
    std::string err;
};

namespace fdtd {

// ---- errors (ctx.cu): the message goes to the context, or to fdtd_last_error(NULL) when c is NULL
extern thread_local std::string g_create_error;
int fail(fdtd_ctx *c, int code, const char *fmt, ...);
int bfail(fdtd_batch *b, int code, const char *fmt, ...);

#define CK(ctx, call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? FDTD_ERR_OOM : FDTD_ERR_CUDA, "%s: %s", #call, \
                        cudaGetErrorString(e_));                                                        \
    } while (0)

// Device memory comes from a library-owned stream-ordered pool per device that keeps freed

// ---- device and driver (ctx.cu)
PFN_cuTensorMapEncodeTiled_v12000 get_encode();
int num_sms();
inline size_t esize(int storage) { return storage == FDTD_F32 ? 4 : 2; }

// ---- stream-ordered device pool with host-side failure injection (pool.cu)
extern std::atomic<int> g_fail_alloc_in;
cudaMemPool_t lib_pool();
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);
cudaError_t dmalloc(fdtd_ctx *c, void **p, size_t bytes);

// ---- context helpers (ctx.cu)
CavityDesc make_desc(const fdtd_ctx *c, int parity_off);
int upload_desc(fdtd_ctx *c);
int encode_maps(fdtd_ctx *c, int set, int box_y);
void drop_graphs(std::map<GraphKey, cudaGraphExec_t> &g);
bool use_fused(const fdtd_ctx *c);
bool use_temporal(const fdtd_ctx *c);
int one_step_kind(const fdtd_ctx *c);
int launch_one(fdtd_ctx *c, int parity, int inject_us, int kind = 0);
int check_status(fdtd_ctx *c, int *d_status, cudaStream_t s);
int ensure_stage(fdtd_ctx *c);
int ensure_stage2(fdtd_ctx *c);

// ---- launch planning (plan.cu)
struct Shape {
    int kind;   // 0: one step per launch, 1: two steps per launch, 2: one fourth-order step, 3: three steps
    int tile_y, stages, ctas_per_sm;
    int rows_per_warp;   // kind 1: rows per consumer warp (1, or 2 for FDTD_KERNEL_TEMPORAL2)
};
// Rows per consumer warp of the two-step kernel a tuning selects.
inline int two_step_rows(const fdtd_tuning &t) { return t.kernel == FDTD_KERNEL_TEMPORAL2 ? 2 : 1; }
Shape resolve_shape(int storage, const fdtd_tuning &t, int kind = 0);
int choose_zlen(long long cols, int nz, int grid, int zchunk, int prologue_planes);
long long simulate_plan(const std::vector<int> &plan, long long cols, int G, int prologue);
std::vector<int> plan_chunks(long long cols, int nz, int G, int prologue, int zchunk);
TileRec base_rec(const fdtd_ctx *c, int parity_off, int set = 0);
void append_tiles_plan(std::vector<TileRec> &v, const fdtd_ctx *c, int parity_off, int tile_y,
                       const std::vector<int> &plan, int kind);
void append_tiles(std::vector<TileRec> &v, const fdtd_ctx *c, int parity_off, int tile_y, int zlen, int kind = 0);
std::vector<TileRec> assign_tiles(const std::vector<TileRec> &v, int G, int prologue, std::vector<int> &first);
int build_tiles(fdtd_ctx *c, int kind);

// ---- z-slabs (slab.cu)
int slab_reach(const fdtd_ctx *c);                 // planes a step's dependence reaches (order 2: 1, order 4: 3)
void slab_after_load(fdtd_ctx *c);                 // a load leaves the ghost cells untrusted
int slab_check_steps(fdtd_ctx *c, int nsteps);     // FDTD_ERR_STATE when the ghosts do not cover nsteps
void slab_took_steps(fdtd_ctx *c, int nsteps);

// ---- point currents and probes (extras_api.cu)
bool extras_on(const fdtd_ctx *c);
int launch_extras_after(fdtd_ctx *c, int copy);

// ---- autotuning (autotune.cu)
int trial_length(int trial_steps);
std::vector<fdtd_tuning> tune_candidates(bool batch, int order = 2);

}  // namespace fdtd
