// C ABI of libfdtd (declared in include/fdtd.h): context lifecycle, layout
// conversion, step dispatch (fused TMA kernel, or the unfused baseline), FP64
// reductions, CUDA-graph replay and batches of cavities.
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

using namespace fdtd;

namespace {

thread_local std::string g_create_error;

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

size_t esize(int storage) { return storage == FDTD_F32 ? 4 : 2; }

struct GraphKey {
    int steps, parity, kind = 0;
    bool operator<(const GraphKey &o) const {
        if (kind != o.kind) return kind < o.kind;
        return steps != o.steps ? steps < o.steps : parity < o.parity;
    }
};

}  // namespace

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
    int maps_by[kMapSets] = {0, 0, 0};      // box height each map set was encoded for (0: not yet)
    CavityDesc *d_desc = nullptr;
    struct TileList {
        TileRec *d = nullptr;   // records, followed by the per-CTA range offsets
        int *first = nullptr;   // inside the same allocation as d
        int n = 0, grid = 0, key = 0;
    } tl[3];                                // [0] one-step, [1] two-step, [2] fourth-order kernel
    int order = 2;                          // spatial order of the differences (2: Eq. 2, 4: the (2,4) scheme)
    double courant = 0.0;                   // max over cells of 3 ce ch (stable for order 2 when <= 1)
    int ch_uniform = 1;
    fdtd_tuning tuning{};
    std::map<GraphKey, cudaGraphExec_t> graphs;
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
    cudaStream_t stream = nullptr;
    std::vector<Member> members;
    long long step = 0;              // step clock: steps enqueued so far (a two-step launch advances it by 2)
    long long launches = 0;          // launches enqueued so far; the next launch has parity launches & 1
    long long *d_step = nullptr;     // device copy of the step clock (advanced by a kernel after each launch)
    fdtd_tuning tuning{};
    TileRec *d_tiles = nullptr;
    int tiles_cap = 0, ntiles = 0, grid = 0;
    bool dirty = true;
    int *d_status = nullptr;
    cudaEvent_t done_ev = nullptr;   // recorded at member removal; the member's stream waits on it
    // Completion marks: after each fdtd_batch_step call, an event and the clock it brings the batch
    // to.  A removed member's stream waits only for the first mark at or past the clock at which the
    // member took its last step (later launches skip it), not for everything enqueued since.
    std::deque<std::pair<long long, cudaEvent_t>> marks;
    std::vector<cudaEvent_t> free_marks;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::vector<cudaGraphExec_t> retired_graphs;   // destroyed at the next synchronisation point
    std::string err;
};

namespace {

int fail(fdtd_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_create_error = buf;
    return code;
}
int bfail(fdtd_batch *b, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return code;
}

#define CK(ctx, call)                                                                                   \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? FDTD_ERR_OOM : FDTD_ERR_CUDA, "%s: %s", #call, \
                        cudaGetErrorString(e_));                                                        \
    } while (0)

// Device memory comes from a library-owned stream-ordered pool per device that keeps freed
// memory for reuse (release threshold: never), so creating and destroying contexts at a
// serving rate neither returns memory to the driver nor synchronises the device.
cudaMemPool_t lib_pool() {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    pools[dev] = pool;
    return pool;
}

// Host-side fault injection (fdtd_debug_fail_alloc): the allocation that counts this down to zero fails.
std::atomic<int> g_fail_alloc_in{-1};

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    for (int n = g_fail_alloc_in.load(); n >= 0;)
        if (g_fail_alloc_in.compare_exchange_weak(n, n - 1)) {
            if (n == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    cudaMemPool_t pool = lib_pool();
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void pool_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

cudaError_t dmalloc(fdtd_ctx *c, void **p, size_t bytes) {
    cudaError_t e = pool_alloc(p, bytes, c->stream);
    if (e == cudaSuccess) c->bytes += (long long)bytes;
    return e;
}

CavityDesc make_desc(const fdtd_ctx *c, int parity_off) {
    CavityDesc d{};
    d.nx = c->nx;
    d.ny = c->ny;
    d.nz = c->nz;
    d.pitch = c->pitch;
    d.plane = (long long)c->pitch * c->ny;
    d.coef_mode = c->coef_mode;
    d.ntab = c->ntab;
    d.parity_off = parity_off;
    for (int q = 0; q < 3; ++q) {
        d.ce[q] = c->ce_s[q];
        d.ch[q] = c->ch_s[q];
        d.face[q] = c->face[q];
        d.face_ch[q] = c->face_ch[q];
    }
    for (int f = 0; f < 6; ++f) {
        d.scale[f] = c->scale[f];
        d.inv_scale[f] = 1.0f / c->scale[f];
        d.buf[0][f] = c->fields[0][f];
        d.buf[1][f] = c->fields[1][f];
        d.coef[f] = c->coef_full[f];
    }
    d.id = c->id;
    d.table = c->table;
    d.inv_table = c->inv_table;
    for (int q = 0; q < 3; ++q) {
        d.inv_ce[q] = 1.0f / c->ce_s[q];
        d.inv_ch[q] = 1.0f / c->ch_s[q];
    }
    d.maps = c->d_maps;
    return d;
}

int upload_desc(fdtd_ctx *c) {
    CavityDesc d = make_desc(c, 0);
    CK(c, cudaMemcpyAsync(c->d_desc, &d, sizeof d, cudaMemcpyHostToDevice, c->stream));
    return FDTD_OK;
}

// Encode the 13 tensor maps of map set `set` (0: one-step kernel, 1: two-step kernel) for
// boxes box_y rows high.  Set 1 sits right after set 0 in the context's map array.
int encode_maps(fdtd_ctx *c, int set, int box_y) {
    if (c->maps_by[set] == box_y) return FDTD_OK;
    auto enc = get_encode();
    if (!enc) return fail(c, FDTD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int hx = 16 / (int)esize(c->storage);
    const int bx = kTileX + 2 * hx;
    std::vector<CUtensorMap> &maps = c->host_maps[set];
    maps.assign(kMapsPerCavity, CUtensorMap{});
    const size_t es = esize(c->storage);
    const CUtensorMapDataType dt = c->storage == FDTD_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : c->storage == FDTD_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint64_t gdim[3] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, (cuuint64_t)c->nz};
    cuuint32_t estr[3] = {1, 1, 1};
    for (int cp = 0; cp < 2; ++cp)
        for (int f = 0; f < 6; ++f) {
            cuuint64_t gstr[2] = {(cuuint64_t)c->pitch * es, (cuuint64_t)c->pitch * c->ny * es};
            cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)box_y, 1};
            CUresult r = enc(&maps[cp * 6 + f], dt, 3, c->fields[cp][f], gdim, gstr, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(c, FDTD_ERR_CUDA, "tensor map encode failed (%d)", (int)r);
        }
    if (set >= 1)   // two-step and fourth-order kernels: slot cp * 6 holds one 4-D map over the six arrays
        for (int cp = 0; cp < 2; ++cp) {
            cuuint64_t gdim4[4] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, (cuuint64_t)c->nz, 6};
            cuuint64_t gstr4[3] = {(cuuint64_t)c->pitch * es, (cuuint64_t)c->pitch * c->ny * es,
                                   (cuuint64_t)c->arr_elems * es};
            cuuint32_t box4[4] = {(cuuint32_t)bx, (cuuint32_t)box_y, 1, 6};
            cuuint32_t estr4[4] = {1, 1, 1, 1};
            CUresult r = enc(&maps[cp * 6], dt, 4, c->fields[cp][0], gdim4, gstr4, box4, estr4,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(c, FDTD_ERR_CUDA, "4-D tensor map encode failed (%d)", (int)r);
        }
    if (c->id) {
        cuuint64_t gstr[2] = {(cuuint64_t)c->pitch, (cuuint64_t)c->pitch * c->ny};
        // ids from 16 bytes left of the tile; the fourth-order kernel also needs its right halo
        cuuint32_t box[3] = {(cuuint32_t)(kTileX + (set == 2 ? 32 : 16)), (cuuint32_t)box_y, 1};
        CUresult r = enc(&maps[12], CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, c->id, gdim, gstr, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(c, FDTD_ERR_CUDA, "id tensor map encode failed (%d)", (int)r);
    }
    CK(c, cudaMemcpyAsync(c->d_maps + set * kMapsPerCavity, maps.data(), sizeof(CUtensorMap) * kMapsPerCavity,
                          cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->maps_by[set] = box_y;
    return FDTD_OK;
}

struct Shape {
    int kind;   // 0: one step per launch, 1: two steps per launch, 2: one fourth-order step
    int tile_y, stages, ctas_per_sm;
};

// Launch shape of kernel kind 0 (one step) or 1 (two steps) from the tuning (invalid fields -> defaults).
Shape resolve_shape(int storage, const fdtd_tuning &t, int kind = 0) {
    static std::mutex mu;
    static std::map<int, int> occ_cache;   // (kind, storage, tile_y, stages) -> max CTAs per SM
    Shape s;
    s.kind = kind;
    if (kind == 2)
        s.tile_y = (t.tile_y == 4 || t.tile_y == 8 || t.tile_y == 12 || t.tile_y == 16) ? t.tile_y : 12;
    else if (kind == 0)
        s.tile_y = (t.tile_y == 4 || t.tile_y == 8 || t.tile_y == 16) ? t.tile_y : 8;
    else
        s.tile_y = (t.tile_y == 8 || t.tile_y == 12 || t.tile_y == 16) ? t.tile_y : 16;
    const int min_st = kind == 2 ? 4 : 3;
    // default ring depths: measured best at 512^3; the fourth-order kernel (three units resident) takes
    // the deepest ring that fits, which measured best for each of its tile heights
    s.stages = (t.stages >= min_st && t.stages <= 8) ? t.stages : (kind == 0 ? 4 : kind == 1 ? 6 : 8);
    auto smem = [&](int st) {
        return kind == 0 ? fused_smem_bytes(storage, s.tile_y, st)
               : kind == 1 ? fused2_smem_bytes(storage, s.tile_y, st)
                           : fused4_smem_bytes(storage, s.tile_y, st);
    };
    while (s.stages > min_st && smem(s.stages) > 227 * 1024) --s.stages;
    const int key = ((kind * 4 + storage) * 64 + s.tile_y) * 16 + s.stages;
    int occ = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = occ_cache.find(key);
        if (it != occ_cache.end()) {
            occ = it->second;
        } else {
            cudaError_t e = kind == 0   ? fused_occupancy(storage, s.tile_y, s.stages, &occ)
                            : kind == 1 ? fused2_occupancy(storage, s.tile_y, s.stages, &occ)
                                        : fused4_occupancy(storage, s.tile_y, s.stages, &occ);
            if (e != cudaSuccess || occ < 1) occ = 1;
            occ_cache[key] = occ;
        }
    }
    s.ctas_per_sm = t.ctas_per_sm > 0 ? std::min(t.ctas_per_sm, occ) : occ;
    return s;
}

// Planes per tile for equal tiles dealt round-robin to `grid` CTAs: fewest plane-times on the
// busiest CTA, counting `prologue_planes` of z-recurrence priming per tile.
int choose_zlen(long long cols, int nz, int grid, int zchunk, int prologue_planes) {
    if (zchunk > 0) return std::min(zchunk, nz);
    long long best = -1;
    int bestL = nz;
    for (int L = nz; L >= 1; --L) {
        const long long nch = (nz + L - 1) / L;
        const long long waves = (cols * nch + grid - 1) / grid;
        const long long cost = waves * (L + prologue_planes);
        if (best < 0 || cost < best) {
            best = cost;
            bestL = L;
        }
    }
    return bestL;
}

// ---------------------------------------------------------------------------------------------
// Work split of one cavity over the persistent CTAs (one CTA per SM).  A tile is a column (tile_x x tile_y cells)
// over a z-chunk of planes and costs (chunk + prologue) plane-times (the prologue planes prime the
// z recurrence); every plane costs the same.  Tiles are listed chunk-major (all columns of chunk 0,
// then chunk 1, ...) so that the tiles running at the same time are neighbours and share their
// halos in L2, and each tile goes to the CTA that becomes free first (greedy list scheduling,
// computed here).  The chunk plan is the one with the shortest simulated makespan among: n equal
// chunks (n = 1..64), and n chunks of length L followed by the rest split into 1-4 pieces.

// Makespan of the greedy schedule of `plan` (chunk lengths) over `cols` columns and G CTAs.
// All tiles of a chunk have one length, so CTAs with equal finish times move together.
long long simulate_plan(const std::vector<int> &plan, long long cols, int G, int prologue) {
    std::map<long long, long long> busy;   // finish time -> number of CTAs
    busy[0] = G;
    for (int len : plan) {
        long long m = cols;
        const long long d = len + prologue;
        while (m > 0) {
            auto it = busy.begin();
            const long long t = it->first, k = std::min(it->second, m);
            if ((it->second -= k) == 0) busy.erase(it);
            busy[t + d] += k;
            m -= k;
        }
    }
    return busy.rbegin()->first;
}

std::vector<int> plan_chunks(long long cols, int nz, int G, int prologue, int zchunk) {
    std::vector<int> plan;
    if (zchunk > 0) {
        for (int z = 0; z < nz; z += zchunk) plan.push_back(std::min(zchunk, nz - z));
        return plan;
    }
    static std::mutex mu;
    static std::map<std::tuple<long long, int, int, int>, std::vector<int>> cache;
    const auto key = std::make_tuple(cols, nz, G, prologue);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    long long best = -1;
    auto consider = [&](const std::vector<int> &p) {
        const long long t = simulate_plan(p, cols, G, prologue);
        if (best < 0 || t < best) {
            best = t;
            plan = p;
        }
    };
    for (int n = 1; n <= std::min(nz, 64); ++n) {   // n nearly equal chunks
        std::vector<int> p;
        for (int q = 0; q < n; ++q) p.push_back(nz / n + (q < nz % n ? 1 : 0));
        consider(p);
    }
    for (int n = 1; n <= std::min(nz, 64); ++n) {   // n chunks of L = nz / (n + 1) .. nz / n, then a split tail
        for (int L = std::max(1, nz / (n + 1)); L <= nz / n; ++L) {
            const int rest = nz - n * L;
            if (rest <= 0) continue;
            for (int pieces = 1; pieces <= std::min(4, rest); ++pieces) {
                std::vector<int> p(n, L);
                for (int q = 0; q < pieces; ++q) p.push_back(rest / pieces + (q < rest % pieces ? 1 : 0));
                consider(p);
            }
        }
    }
    std::lock_guard<std::mutex> g(mu);
    cache[key] = plan;
    return plan;
}

TileRec base_rec(const fdtd_ctx *c, int parity_off, int set = 0) {
    TileRec r{};
    r.nx = c->nx;
    r.ny = c->ny;
    r.nz = c->nz;
    r.pitch = c->pitch;
    r.mode = c->coef_mode;
    r.plane = (long long)c->pitch * c->ny;
    r.ch_uniform = c->ch_uniform;
    r.parity_off = parity_off;
    const float re = c->scale[0] / c->scale[3];   // s_E / s_H (1 for FP32)
    for (int q = 0; q < 3; ++q) {
        r.ce[q] = c->ce_s[q] * re;
        r.ch[q] = c->ch_s[q] / re;
    }
    r.table = reinterpret_cast<const float4 *>(c->table_fused);
    r.ntab = c->ntab;
    r.stop = LLONG_MAX;
    r.maps = c->d_maps + set * kMapsPerCavity;
    for (int f = 0; f < 6; ++f) {
        r.dst[0][f] = c->fields[0][f];
        r.dst[1][f] = c->fields[1][f];
    }
    return r;
}

// Tiles of the one-step kernel (kind 0: 64 cells wide) or the two-step kernel (kind 1: W wide),
// chunk-major over the z-chunks of `plan`.
void append_tiles_plan(std::vector<TileRec> &v, const fdtd_ctx *c, int parity_off, int tile_y,
                       const std::vector<int> &plan, int kind) {
    const TileRec b = base_rec(c, parity_off, kind);
    const int tw = kind == 1 ? fused2_tile_w(c->storage) : kTileX;
    int z0 = 0;
    for (int len : plan) {
        for (int y0 = 0; y0 < c->ny; y0 += tile_y)
            for (int x0 = 0; x0 < c->nx; x0 += tw) {
                TileRec t = b;
                t.x0 = x0;
                t.y0 = y0;
                t.kz0 = z0;
                t.kz1 = z0 + len;
                t.id_x0 = (x0 - 2) & ~15;   // two-step kernel: 16-byte aligned origin of the id box
                v.push_back(t);
            }
        z0 += len;
    }
}

void append_tiles(std::vector<TileRec> &v, const fdtd_ctx *c, int parity_off, int tile_y, int zlen, int kind = 0) {
    std::vector<int> plan;
    for (int z = 0; z < c->nz; z += zlen) plan.push_back(std::min(zlen, c->nz - z));
    append_tiles_plan(v, c, parity_off, tile_y, plan, kind);
}

// Greedy assignment of the listed tiles to G CTAs (each tile to the CTA that frees first, lowest
// index on ties); returns the tiles regrouped by CTA and, in first, each CTA's range (G + 1 entries).
std::vector<TileRec> assign_tiles(const std::vector<TileRec> &v, int G, int prologue, std::vector<int> &first) {
    using Slot = std::pair<long long, int>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> q;
    for (int b = 0; b < G; ++b) q.push({0, b});
    std::vector<std::vector<int>> per(G);
    for (int i = 0; i < (int)v.size(); ++i) {
        const Slot sl = q.top();
        q.pop();
        per[sl.second].push_back(i);
        q.push({sl.first + (v[i].kz1 - v[i].kz0) + prologue, sl.second});
    }
    std::vector<TileRec> out;
    out.reserve(v.size());
    first.assign(G + 1, 0);
    for (int b = 0; b < G; ++b) {
        first[b] = (int)out.size();
        for (int i : per[b]) out.push_back(v[i]);
    }
    first[G] = (int)out.size();
    return out;
}

int build_tiles(fdtd_ctx *c, int kind) {
    Shape s = resolve_shape(c->storage, c->tuning, kind);
    fdtd_ctx::TileList &tl = c->tl[kind];
    if (tl.key == s.tile_y && tl.d && tl.grid) return FDTD_OK;
    int rc = encode_maps(c, kind, s.tile_y + (kind == 0 ? 2 : kind == 1 ? 4 : 6));
    if (rc) return rc;
    const int tw = kind == 1 ? fused2_tile_w(c->storage) : kTileX;
    const long long cols = (long long)((c->nx + tw - 1) / tw) * ((c->ny + s.tile_y - 1) / s.tile_y);
    const int prologue = kind == 0 ? 1 : kind == 1 ? 3 : 4;
    const int G = (int)std::min<long long>((long long)num_sms() * s.ctas_per_sm, cols * c->nz);
    std::vector<TileRec> listed, v;
    std::vector<int> first;
    int grid;
    if (s.ctas_per_sm == 1) {
        // one CTA per SM: CTAs run at the same rate, so the greedy schedule is what the SMs see
        append_tiles_plan(listed, c, 0, s.tile_y, plan_chunks(cols, c->nz, G, prologue, c->tuning.zchunk), kind);
        grid = (int)std::min<size_t>(listed.size(), (size_t)G);
        v = assign_tiles(listed, grid, prologue, first);
    } else {
        // co-resident CTAs share their SM's issue slots: equal tiles in round-robin waves
        append_tiles(v, c, 0, s.tile_y, choose_zlen(cols, c->nz, G, c->tuning.zchunk, prologue), kind);
        grid = (int)std::min<size_t>(v.size(), (size_t)G);
    }
    pool_free(tl.d, c->stream);
    tl.d = nullptr;
    // tile records, then the grid + 1 range offsets (16-byte aligned after the 256-byte records)
    const size_t rec_bytes = sizeof(TileRec) * v.size();
    CK(c, pool_alloc((void **)&tl.d, rec_bytes + sizeof(int) * first.size(), c->stream));
    CK(c, cudaMemcpyAsync(tl.d, v.data(), rec_bytes, cudaMemcpyHostToDevice, c->stream));
    tl.first = nullptr;
    if (!first.empty()) {
        tl.first = reinterpret_cast<int *>(reinterpret_cast<char *>(tl.d) + rec_bytes);
        CK(c, cudaMemcpyAsync(tl.first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice,
                              c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    tl.n = (int)v.size();
    tl.grid = grid;
    tl.key = s.tile_y;
    return FDTD_OK;
}

void drop_graphs(std::map<GraphKey, cudaGraphExec_t> &g) {
    for (auto &kv : g) cudaGraphExecDestroy(kv.second);
    g.clear();
}

bool use_fused(const fdtd_ctx *c) {
    return c->coef_mode != COEF_FULL && c->tuning.kernel != FDTD_KERNEL_SIMPLE;
}

// AUTO takes the two-step kernel: faster than the one-step kernel at every size measured (second
// order only: the fourth-order scheme has a one-step kernel)
bool use_temporal(const fdtd_ctx *c) {
    return use_fused(c) && c->order == 2 &&
           (c->tuning.kernel == FDTD_KERNEL_TEMPORAL || c->tuning.kernel == FDTD_KERNEL_AUTO);
}

// Tile kind of a context's one-step launches: 0 (Eq. 2) or 2 (fourth order).
int one_step_kind(const fdtd_ctx *c) { return c->order == 4 ? 2 : 0; }

// One launch of a single context (no graph): kinds 0 and 2 advance one step, kind 1 two steps.
int launch_one(fdtd_ctx *c, int parity, int inject_us, int kind = 0) {
    if (!use_fused(c)) {
        if (c->order == 4)
            CK(c, launch_simple4_step(c->storage, make_desc(c, 0), c->cur, c->stream));
        else
            CK(c, launch_simple_step(c->storage, make_desc(c, 0), c->cur, c->stream));
        return FDTD_OK;
    }
    Shape s = resolve_shape(c->storage, c->tuning, kind);
    const fdtd_ctx::TileList &tl = c->tl[kind];
    FusedLaunch L{};
    L.recs = tl.d;
    L.ntiles = tl.n;
    L.parity = parity;
    L.status = c->d_status;
    L.tile_y = s.tile_y;
    L.stages = s.stages;
    L.grid = tl.grid;
    L.inject_timeout_us = inject_us;
    L.first = tl.first;
    if (kind == 0)
        CK(c, launch_fused_step(c->storage, L, c->stream));
    else if (kind == 1)
        CK(c, launch_fused2_step(c->storage, L, c->stream));
    else
        CK(c, launch_fused4_step(c->storage, L, c->stream));
    return FDTD_OK;
}

bool extras_on(const fdtd_ctx *c) { return c->nsrc > 0 || c->nprobe > 0; }

// The point-current / probe launch after a step that left the state in copy `copy`.
int launch_extras_after(fdtd_ctx *c, int copy) {
    ExtrasParams X{};
    X.clock = c->d_xclock;
    X.nsrc = c->nsrc;
    X.wave_len = c->wave_len;
    X.src_comp = c->d_src_comp;
    X.src_off = c->d_src_off;
    X.wave = c->d_wave;
    X.dx = (float)c->dx;
    X.nprobe = c->nprobe;
    X.capacity = c->probe_cap;
    X.probe_start = c->probe_start;
    X.probe_comp = c->d_probe_comp;
    X.probe_off = c->d_probe_off;
    X.probe_buf = c->d_probe_buf;
    CK(c, launch_extras(c->storage, make_desc(c, 0), copy, X, c->stream));
    return FDTD_OK;
}

int check_status(fdtd_ctx *c, int *d_status, cudaStream_t s) {
    int h = 0;
    CK(c, cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    if (h) {
        CK(c, cudaMemsetAsync(d_status, 0, sizeof(int), s));
        CK(c, cudaStreamSynchronize(s));
        if (h & STATUS_TIMEOUT)
            return fail(c, FDTD_ERR_TIMEOUT, "a step kernel's bounded wait ran out (status 0x%x)", h);
        return fail(c, FDTD_ERR_CUDA, "device status 0x%x", h);
    }
    return FDTD_OK;
}

int ensure_stage(fdtd_ctx *c) {
    if (c->d_stage) return FDTD_OK;
    const size_t n = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
    CK(c, dmalloc(c, (void **)&c->d_stage, n * sizeof(float)));
    return FDTD_OK;
}

// Two staging buffers, a copy stream and its events for pipelined host loads.
int ensure_stage2(fdtd_ctx *c) {
    if (int rc = ensure_stage(c)) return rc;
    if (c->d_stage2) return FDTD_OK;
    const size_t n = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
    CK(c, dmalloc(c, (void **)&c->d_stage2, n * sizeof(float)));
    CK(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        CK(c, cudaEventCreateWithFlags(&c->staged[b], cudaEventDisableTiming));
        CK(c, cudaEventCreateWithFlags(&c->packed[b], cudaEventDisableTiming));
    }
    return FDTD_OK;
}

// Compress per-position coefficients: one byte per active cell + table when <= 256 distinct tuples.
struct Tuple {
    float v[6];
    bool operator==(const Tuple &o) const { return memcmp(v, o.v, sizeof v) == 0; }
};
struct TupleHash {
    size_t operator()(const Tuple &t) const {
        uint64_t h = 1469598103934665603ull;
        const unsigned char *p = reinterpret_cast<const unsigned char *>(t.v);
        for (size_t i = 0; i < sizeof t.v; ++i) h = (h ^ p[i]) * 1099511628211ull;
        return (size_t)h;
    }
};

}  // namespace

namespace fdtd {
// Message returned by fdtd_last_error(NULL) on this thread (used by context-free entry points).
void set_last_error(const char *msg) { g_create_error = msg; }
}  // namespace fdtd

extern "C" {

const char *fdtd_version(void) { return "fdtd-gb300 0.1 (sm_103a)"; }

const char *fdtd_last_error(const fdtd_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int fdtd_create(fdtd_ctx **out, int nx, int ny, int nz, double dt, double dx, const float *const ce[3],
                const float *const ch[3], int storage, void *cuda_stream) {
    if (!out) return fail(nullptr, FDTD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 32768 || ny > 32768 || nz > 32768)
        return fail(nullptr, FDTD_ERR_ARG, "cell counts must be in [1, 32768], got %d x %d x %d", nx, ny, nz);
    if (!(dt > 0) || !(dx > 0) || !std::isfinite(dt) || !std::isfinite(dx))
        return fail(nullptr, FDTD_ERR_ARG, "dt and dx must be positive and finite");
    if (storage < FDTD_F32 || storage > FDTD_BF16) return fail(nullptr, FDTD_ERR_ARG, "bad storage %d", storage);
    bool have_ce = ce && ce[0] && ce[1] && ce[2];
    bool have_ch = ch && ch[0] && ch[1] && ch[2];
    if ((ce && !have_ce && (ce[0] || ce[1] || ce[2])) || (ch && !have_ch && (ch[0] || ch[1] || ch[2])))
        return fail(nullptr, FDTD_ERR_ARG, "coefficient arrays must be all three or none");

    const size_t CX = nx + 1, CY = ny + 1;
    auto cidx = [&](int i, int j, int k) { return ((size_t)k * CY + j) * CX + i; };
    const float vac = (float)(dt / dx);

    // ---- coefficient validation, Courant check and compression (host)
    std::vector<uint8_t> ids;
    std::vector<Tuple> table;
    bool full = false;
    double courant = 3.0 * vac * vac;   // max over cells of 3 ce ch
    if (have_ce || have_ch) {
        ids.resize((size_t)nx * ny * nz);
        std::unordered_map<Tuple, int, TupleHash> map;
        Tuple last{};
        int last_id = -1;
        double worst = 0.0;
        for (int k = 0; k < nz && !full; ++k)
            for (int j = 0; j < ny && !full; ++j)
                for (int i = 0; i < nx; ++i) {
                    Tuple t;
                    const size_t q = cidx(i, j, k);
                    for (int c = 0; c < 3; ++c) {
                        t.v[c] = have_ce ? ce[c][q] : vac;
                        t.v[3 + c] = have_ch ? ch[c][q] : vac;
                    }
                    int id;
                    if (last_id >= 0 && t == last) {
                        id = last_id;
                    } else {
                        for (int c = 0; c < 6; ++c)
                            if (!(t.v[c] > 0.f) || !std::isfinite(t.v[c]))
                                return fail(nullptr, FDTD_ERR_ARG, "coefficient %d at (%d,%d,%d) is not positive", c,
                                            i, j, k);
                        const double me = std::max({t.v[0], t.v[1], t.v[2]});
                        const double mh = std::max({t.v[3], t.v[4], t.v[5]});
                        worst = std::max(worst, 3.0 * me * mh);
                        auto it = map.find(t);
                        if (it == map.end()) {
                            if ((int)table.size() >= kMaxTable) {
                                full = true;
                                break;
                            }
                            id = (int)table.size();
                            map.emplace(t, id);
                            table.push_back(t);
                        } else {
                            id = it->second;
                        }
                        last = t;
                        last_id = id;
                    }
                    ids[((size_t)k * ny + j) * nx + i] = (uint8_t)id;
                }
        if (full) {
            // per-position arrays: validate and Courant-check every active cell
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        const size_t q = cidx(i, j, k);
                        double me = 0, mh = 0;
                        for (int c = 0; c < 3; ++c) {
                            const float a = have_ce ? ce[c][q] : vac, b = have_ch ? ch[c][q] : vac;
                            if (!(a > 0.f) || !(b > 0.f) || !std::isfinite(a) || !std::isfinite(b))
                                return fail(nullptr, FDTD_ERR_ARG, "coefficient at (%d,%d,%d) is not positive", i,
                                            j, k);
                            me = std::max(me, (double)a);
                            mh = std::max(mh, (double)b);
                        }
                        worst = std::max(worst, 3.0 * me * mh);
                    }
        }
        if (worst > 1.0 + 1e-6)
            return fail(nullptr, FDTD_ERR_UNSTABLE, "Courant bound violated: max sqrt(3 ce ch) = %.6f > 1",
                        std::sqrt(worst));
        courant = worst;
        // far-face ch values (Hx at i = nx, Hy at j = ny, Hz at k = nz) are used by energy and divergence
        if (have_ch) {
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j <= ny; ++j)
                    for (int i = 0; i <= nx; ++i) {
                        const bool fx = i == nx && j < ny, fy = j == ny && i < nx;
                        if ((fx && !(ch[0][cidx(i, j, k)] > 0.f)) || (fy && !(ch[1][cidx(i, j, k)] > 0.f)))
                            return fail(nullptr, FDTD_ERR_ARG, "ch on a far face is not positive");
                    }
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i)
                    if (!(ch[2][cidx(i, j, nz)] > 0.f)) return fail(nullptr, FDTD_ERR_ARG, "chz on face k=nz not positive");
        }
    } else {
        if (3.0 * vac * vac > 1.0 + 1e-6)
            return fail(nullptr, FDTD_ERR_UNSTABLE, "Courant bound violated: sqrt(3) dt/dx = %.6f > 1",
                        std::sqrt(3.0) * vac);
    }

    fdtd_ctx *c = new fdtd_ctx();
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->dt = dt;
    c->dx = dx;
    c->courant = courant;
    c->storage = storage;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->pitch = (nx + 31) / 32 * 32;
    c->arr_elems = (size_t)c->pitch * ny * nz;
    for (int q = 0; q < 3; ++q) c->ce_s[q] = c->ch_s[q] = vac;
    auto bail = [&](int code) {
        fdtd_destroy(c);
        return code;
    };
    auto cfail = [&](const char *what, cudaError_t e) {
        fail(nullptr, e == cudaErrorMemoryAllocation ? FDTD_ERR_OOM : FDTD_ERR_CUDA, "%s: %s", what,
             cudaGetErrorString(e));
        return bail(e == cudaErrorMemoryAllocation ? FDTD_ERR_OOM : FDTD_ERR_CUDA);
    };
    cudaError_t e;
    const size_t es = esize(storage);
    // each copy's six arrays in one allocation, arr_elems apart, so that one 4-D tensor map (x, y, z,
    // field) covers all of them (the two-step kernel loads a unit's six boxes with one TMA instruction)
    for (int cp = 0; cp < 2; ++cp) {
        if ((e = dmalloc(c, &c->fields[cp][0], 6 * c->arr_elems * es)) != cudaSuccess) return cfail("field alloc", e);
        if ((e = cudaMemsetAsync(c->fields[cp][0], 0, 6 * c->arr_elems * es, c->stream)) != cudaSuccess)
            return cfail("memset", e);
        for (int f = 1; f < 6; ++f) c->fields[cp][f] = static_cast<char *>(c->fields[cp][0]) + f * c->arr_elems * es;
    }
    const size_t nface[3] = {(size_t)ny * nz, (size_t)nx * nz, (size_t)nx * ny};
    for (int q = 0; q < 3; ++q) {
        if ((e = dmalloc(c, (void **)&c->face[q], nface[q] * 4)) != cudaSuccess) return cfail("face alloc", e);
        if ((e = cudaMemsetAsync(c->face[q], 0, nface[q] * 4, c->stream)) != cudaSuccess) return cfail("memset", e);
    }
    if (have_ce || have_ch) {
        // face ch (Hx at i = nx, Hy at j = ny, Hz at k = nz)
        for (int q = 0; q < 3; ++q) {
            std::vector<float> fc(nface[q]);
            for (size_t n = 0; n < nface[q]; ++n) {
                size_t src;
                if (q == 0) src = cidx(nx, (int)(n % ny), (int)(n / ny));
                else if (q == 1) src = cidx((int)(n % nx), ny, (int)(n / nx));
                else src = cidx((int)(n % nx), (int)(n / nx), nz);
                fc[n] = have_ch ? ch[q][src] : vac;
            }
            if ((e = dmalloc(c, (void **)&c->face_ch[q], nface[q] * 4)) != cudaSuccess) return cfail("face alloc", e);
            if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cfail("sync", e);
            if ((e = cudaMemcpy(c->face_ch[q], fc.data(), nface[q] * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
                return cfail("face copy", e);
        }
        if (!full) {
            c->coef_mode = COEF_ID8;
            c->ntab = (int)table.size();
            // ch identical in every cell (per component): the fused kernel then skips its ch lookups
            c->ch_uniform = 1;
            for (int n = 1; n < c->ntab; ++n)
                for (int q = 0; q < 3; ++q)
                    if (table[n].v[3 + q] != table[0].v[3 + q]) c->ch_uniform = 0;
            if (c->ch_uniform)
                for (int q = 0; q < 3; ++q) c->ch_s[q] = table[0].v[3 + q];
            std::vector<float> tab(8 * kMaxTable, 0.f);
            for (int n = 0; n < c->ntab; ++n) {
                for (int q = 0; q < 3; ++q) {
                    tab[8 * n + q] = table[n].v[q];
                    tab[8 * n + 4 + q] = table[n].v[3 + q];
                }
            }
            if ((e = dmalloc(c, (void **)&c->table, tab.size() * 4)) != cudaSuccess) return cfail("table alloc", e);
            if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cfail("sync", e);
            if ((e = cudaMemcpy(c->table, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
                return cfail("table copy", e);
            if ((e = dmalloc(c, (void **)&c->table_fused, tab.size() * 4)) != cudaSuccess)
                return cfail("table alloc", e);
            if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cfail("sync", e);
            if ((e = cudaMemcpy(c->table_fused, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
                return cfail("table copy", e);
            c->host_table = tab;
            std::vector<float> inv(tab.size(), 0.f);
            for (int n = 0; n < c->ntab; ++n)
                for (int q = 0; q < 3; ++q) {
                    inv[8 * n + q] = (float)(1.0 / (double)tab[8 * n + q]);
                    inv[8 * n + 4 + q] = (float)(1.0 / (double)tab[8 * n + 4 + q]);
                }
            if ((e = dmalloc(c, (void **)&c->inv_table, inv.size() * 4)) != cudaSuccess) return cfail("table alloc", e);
            if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cfail("sync", e);
            if ((e = cudaMemcpy(c->inv_table, inv.data(), inv.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
                return cfail("table copy", e);
            if ((e = dmalloc(c, (void **)&c->id, c->arr_elems)) != cudaSuccess) return cfail("id alloc", e);
            if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cfail("sync", e);
            if ((e = cudaMemset(c->id, 0, c->arr_elems)) != cudaSuccess) return cfail("memset", e);
            if ((e = cudaMemcpy2D(c->id, c->pitch, ids.data(), nx, nx, (size_t)ny * nz, cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return cfail("id copy", e);
        } else {
            c->coef_mode = COEF_FULL;
            std::vector<float> row((size_t)c->pitch * ny * nz, 0.f);
            for (int a = 0; a < 6; ++a) {
                for (int k = 0; k < nz; ++k)
                    for (int j = 0; j < ny; ++j)
                        for (int i = 0; i < nx; ++i) {
                            const size_t q = cidx(i, j, k);
                            const float v = a < 3 ? (have_ce ? ce[a][q] : vac) : (have_ch ? ch[a - 3][q] : vac);
                            row[((size_t)k * ny + j) * c->pitch + i] = v;
                        }
                if ((e = dmalloc(c, (void **)&c->coef_full[a], row.size() * 4)) != cudaSuccess)
                    return cfail("coef alloc", e);
                if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cfail("sync", e);
                if ((e = cudaMemcpy(c->coef_full[a], row.data(), row.size() * 4, cudaMemcpyHostToDevice)) !=
                    cudaSuccess)
                    return cfail("coef copy", e);
            }
        }
    }
    if ((e = dmalloc(c, (void **)&c->d_status, sizeof(int))) != cudaSuccess) return cfail("status alloc", e);
    if ((e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream)) != cudaSuccess) return cfail("memset", e);
    const int nb = reduction_blocks();
    if ((e = dmalloc(c, (void **)&c->d_partial, sizeof(double) * 3 * nb)) != cudaSuccess) return cfail("alloc", e);
    if ((e = dmalloc(c, (void **)&c->d_out, sizeof(double) * 3)) != cudaSuccess) return cfail("alloc", e);
    if ((e = dmalloc(c, (void **)&c->d_max, sizeof(unsigned) * 6)) != cudaSuccess) return cfail("alloc", e);
    if ((e = dmalloc(c, (void **)&c->d_maps, sizeof(CUtensorMap) * kMapsPerCavity * kMapSets)) != cudaSuccess)
        return cfail("alloc", e);
    if ((e = dmalloc(c, (void **)&c->d_desc, sizeof(CavityDesc))) != cudaSuccess) return cfail("alloc", e);
    if (int rc = upload_desc(c)) {
        g_create_error = c->err;
        return bail(rc);
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cfail("sync", e);
    *out = c;
    return FDTD_OK;
}

void fdtd_destroy(fdtd_ctx *c) {
    if (!c) return;
    if (c->batch) fdtd_batch_remove(c->batch, c);
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);   // a prefetch may still be copying
    cudaStreamSynchronize(c->stream);
    drop_graphs(c->graphs);
    cudaStream_t st = c->stream;
    for (int cp = 0; cp < 2; ++cp)
        pool_free(c->fields[cp][0], st);   // the six arrays share one allocation
    for (int q = 0; q < 3; ++q) {
        pool_free(c->face[q], st);
        pool_free(c->face_ch[q], st);
    }
    for (int a = 0; a < 6; ++a) pool_free(c->coef_full[a], st);
    for (void *p : {(void *)c->id, (void *)c->table, (void *)c->inv_table, (void *)c->table_fused,
                    (void *)c->d_status, (void *)c->d_partial, (void *)c->d_out, (void *)c->d_stage,
                    (void *)c->d_max, (void *)c->d_maps, (void *)c->d_desc, (void *)c->tl[0].d,
                    (void *)c->tl[1].d, (void *)c->tl[2].d, (void *)c->d_src_comp, (void *)c->d_src_off, (void *)c->d_wave,
                    (void *)c->d_probe_comp, (void *)c->d_probe_off, (void *)c->d_probe_buf, (void *)c->d_xclock})
        pool_free(p, st);
    pool_free(c->d_stage2, st);
    pool_free(c->d_prefetch, st);
    cudaStreamSynchronize(st);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    for (int b = 0; b < 2; ++b) {
        if (c->staged[b]) cudaEventDestroy(c->staged[b]);
        if (c->packed[b]) cudaEventDestroy(c->packed[b]);
    }
    if (c->prefetched) cudaEventDestroy(c->prefetched);
    if (c->prefetch_free) cudaEventDestroy(c->prefetch_free);
    delete c;
}

long long fdtd_steps_done(const fdtd_ctx *c) { return c ? c->steps : -1; }
long long fdtd_device_bytes(const fdtd_ctx *c) { return c ? c->bytes : -1; }

int fdtd_set_tuning(fdtd_ctx *c, const fdtd_tuning *t) {
    if (!c) return FDTD_ERR_ARG;
    fdtd_tuning n{};
    if (t) n = *t;
    if (n.kernel < 0 || n.kernel > FDTD_KERNEL_TEMPORAL) return fail(c, FDTD_ERR_ARG, "bad kernel %d", n.kernel);
    if (n.kernel == FDTD_KERNEL_TEMPORAL && c->order != 2)
        return fail(c, FDTD_ERR_ARG, "the two-step kernel runs the second-order scheme only");
    // one-step kernels: 4, 8 or 16 rows (the fourth-order kernel also 12); two-step kernel: 8, 12 or 16
    const bool ty_one = n.tile_y == 4 || n.tile_y == 8 || n.tile_y == 16 || (c->order == 4 && n.tile_y == 12),
               ty_two = n.tile_y == 8 || n.tile_y == 12 || n.tile_y == 16;
    if (n.tile_y && !(n.kernel == FDTD_KERNEL_TEMPORAL ? ty_two
                      : n.kernel == FDTD_KERNEL_AUTO   ? (ty_one || ty_two)
                                                       : ty_one))
        return fail(c, FDTD_ERR_ARG, "tile_y must be 4, 8 or 16 (fourth order: also 12; two-step kernel: 8, 12 or 16)");
    if (n.stages && (n.stages < 3 || n.stages > 8)) return fail(c, FDTD_ERR_ARG, "stages must be in [3, 8]");
    if (n.stages == 3 && c->order == 4) return fail(c, FDTD_ERR_ARG, "the fourth-order kernel needs stages >= 4");
    if (n.zchunk < 0 || n.ctas_per_sm < 0) return fail(c, FDTD_ERR_ARG, "negative tuning value");
    c->tuning = n;
    c->tl[0].key = c->tl[1].key = c->tl[2].key = 0;   // force tile rebuilds
    cudaStreamSynchronize(c->stream);   // no graph of this context may still be running
    drop_graphs(c->graphs);
    return FDTD_OK;
}

int fdtd_set_order(fdtd_ctx *c, int order) {
    if (!c) return FDTD_ERR_ARG;
    if (order != 2 && order != 4) return fail(c, FDTD_ERR_ARG, "order must be 2 or 4");
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member");
    // the (2,4) difference has symbol up to c1 - c2 = 7/6 times the second-order one
    const double gain = order == 4 ? 7.0 / 6.0 : 1.0;
    if (c->courant * gain * gain > 1.0 + 1e-6)
        return fail(c, FDTD_ERR_UNSTABLE, "Courant bound of order %d violated: max sqrt(3 ce ch) * %.4f = %.6f > 1",
                    order, gain, std::sqrt(c->courant) * gain);
    if (order == 4 && c->tuning.kernel == FDTD_KERNEL_TEMPORAL)
        return fail(c, FDTD_ERR_ARG, "the two-step kernel runs the second-order scheme only; retune first");
    if (order == 4 && c->tuning.stages == 3)
        return fail(c, FDTD_ERR_ARG, "the fourth-order kernel needs stages >= 4; retune first");
    cudaStreamSynchronize(c->stream);   // no graph of this context may still be running
    drop_graphs(c->graphs);
    c->order = order;
    return FDTD_OK;
}

int fdtd_get_order(const fdtd_ctx *c) { return c ? c->order : -1; }

// ---------------------------------------------------------------------------------------------
// Autotuning: candidates are timed on the caller's own state, which is copied aside and restored.
namespace {

std::vector<fdtd_tuning> tune_candidates(bool batch, int order = 2) {
    std::vector<fdtd_tuning> v;
    if (order == 4) {   // the fused fourth-order kernel's tile heights, deepest ring that fits (0) or 4 slots
        for (int ty : {4, 8, 12, 16})
            for (int st : {0, 4}) v.push_back(fdtd_tuning{FDTD_KERNEL_FUSED, ty, 0, 0, st, 1});
        return v;
    }
    for (int ty : {4, 8, 16}) v.push_back(fdtd_tuning{FDTD_KERNEL_FUSED, ty, 0, 0, 4, 1});
    for (int ty : {8, 12, 16})
        for (int st : {4, 6}) {
            if (batch && st != 4) continue;
            v.push_back(fdtd_tuning{FDTD_KERNEL_TEMPORAL, ty, 0, 0, st, 1});
        }
    return v;
}

int trial_length(int trial_steps) {   // whole 16-step graphs
    const int n = trial_steps <= 0 ? 16 : trial_steps;
    return (n + 15) / 16 * 16;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int>, std::pair<fdtd_tuning, double>> g_tune_cache;

}  // namespace

int fdtd_autotune(fdtd_ctx *c, int trial_steps, fdtd_tuning *out, double *ms_per_step) {
    NvtxRange nvtx_range("fdtd_autotune");
    if (!c) return FDTD_ERR_ARG;
    if (!c->has_fields) return fail(c, FDTD_ERR_STATE, "fdtd_set_fields has not been called");
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member; tune the batch");
    if (extras_on(c)) return fail(c, FDTD_ERR_STATE, "tune before setting currents or probes");
    auto report = [&](const fdtd_tuning &t, double ms) {
        if (out) *out = t;
        if (ms_per_step) *ms_per_step = ms;
        return FDTD_OK;
    };
    if (c->coef_mode == COEF_FULL) {   // per-position coefficient arrays: only the unfused kernel applies
        fdtd_tuning t{FDTD_KERNEL_SIMPLE, 0, 0, 0, 0, c->tuning.use_graph};
        if (int rc = fdtd_set_tuning(c, &t)) return rc;
        return report(t, -1.0);
    }
    const auto key = std::make_tuple(c->nx, c->ny, c->nz, c->storage, c->coef_mode, c->ch_uniform, c->order);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            if (int rc = fdtd_set_tuning(c, &it->second.first)) return rc;
            return report(it->second.first, it->second.second);
        }
    }
    const int n = trial_length(trial_steps);
    const size_t bytes = (size_t)c->pitch * c->ny * c->nz * esize(c->storage);
    char *snap = nullptr;
    CK(c, cudaStreamSynchronize(c->stream));
    if (pool_alloc((void **)&snap, 6 * bytes, c->stream) != cudaSuccess)
        return fail(c, FDTD_ERR_OOM, "autotune: no room for a copy of the fields");
    const int cur0 = c->cur;
    const long long steps0 = c->steps;
    for (int f = 0; f < 6; ++f)
        CK(c, cudaMemcpyAsync(snap + f * bytes, c->fields[cur0][f], bytes, cudaMemcpyDeviceToDevice, c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    fdtd_tuning best{};
    double best_ms = -1.0;
    int rc = FDTD_OK;
    for (const fdtd_tuning &t : tune_candidates(false, c->order)) {
        if ((rc = fdtd_set_tuning(c, &t)) != FDTD_OK) break;
        if ((rc = fdtd_step(c, n)) != FDTD_OK) break;   // untimed: tiles, maps and graphs are built here
        cudaEventRecord(e0, c->stream);
        if ((rc = fdtd_step(c, n)) != FDTD_OK) break;
        cudaEventRecord(e1, c->stream);
        if ((rc = fdtd_sync(c)) != FDTD_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / n;
        if (best_ms < 0 || per < best_ms) {
            best_ms = per;
            best = t;
        }
    }
    // put the state back whatever happened
    cudaStreamSynchronize(c->stream);
    for (int f = 0; f < 6; ++f)
        cudaMemcpyAsync(c->fields[cur0][f], snap + f * bytes, bytes, cudaMemcpyDeviceToDevice, c->stream);
    pool_free(snap, c->stream);
    cudaStreamSynchronize(c->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->cur = cur0;
    c->steps = steps0;
    if (rc != FDTD_OK) return rc;
    if (int r2 = fdtd_set_tuning(c, &best)) return r2;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = {best, best_ms};
    }
    return report(best, best_ms);
}

int fdtd_set_fields(fdtd_ctx *c, const float *const f[6], int on_device) {
    NvtxRange nvtx_range("fdtd_set_fields");
    if (!c || !f) return fail(c, FDTD_ERR_ARG, "NULL argument");
    for (int q = 0; q < 6; ++q)
        if (!f[q]) return fail(c, FDTD_ERR_ARG, "field %d is NULL", q);
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member; remove it first");
    const size_t n = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
    if (!on_device)
        if (int rc = ensure_stage(c)) return rc;
    // scales for 16-bit storage: s_c = 2^(8 - ceil(log2 max|F_c|))
    if (c->storage != FDTD_F32) {
        CK(c, cudaMemsetAsync(c->d_max, 0, sizeof(unsigned) * 6, c->stream));
        for (int q = 0; q < 6; ++q) {
            const float *src = f[q];
            if (!on_device) {
                CK(c, cudaMemcpyAsync(c->d_stage, f[q], n * 4, cudaMemcpyHostToDevice, c->stream));
                src = c->d_stage;
            }
            CK(c, launch_maxabs(src, q, c->nx, c->ny, c->nz, c->d_max + q, c->stream));
        }
        unsigned hm[6];
        CK(c, cudaMemcpyAsync(hm, c->d_max, sizeof hm, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        // one power-of-two scale for the three E components and one for the three H components
        for (int g = 0; g < 2; ++g) {
            float mx = 0.f;
            for (int q = 3 * g; q < 3 * g + 3; ++q) {
                float m;
                memcpy(&m, &hm[q], 4);
                if (!std::isfinite(m)) return fail(c, FDTD_ERR_ARG, "field %d holds a non-finite value", q);
                mx = std::max(mx, m);
            }
            const float sc = mx > 0.f ? std::ldexp(1.0f, 8 - (int)std::ceil(std::log2((double)mx))) : 1.0f;
            for (int q = 3 * g; q < 3 * g + 3; ++q) c->scale[q] = sc;
        }
        if (c->table_fused) {
            const float re = c->scale[0] / c->scale[3];
            std::vector<float> tf = c->host_table;
            for (int n = 0; n < c->ntab; ++n)
                for (int q = 0; q < 3; ++q) {
                    tf[8 * n + q] = c->host_table[8 * n + q] * re;
                    tf[8 * n + 4 + q] = c->host_table[8 * n + 4 + q] / re;
                }
            CK(c, cudaMemcpyAsync(c->table_fused, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice, c->stream));
            CK(c, cudaStreamSynchronize(c->stream));
        }
        c->tl[0].key = c->tl[1].key = c->tl[2].key = 0;   // tile records embed the folded coefficients
        cudaStreamSynchronize(c->stream);
        drop_graphs(c->graphs);
    }
    if (int rc = upload_desc(c)) return rc;
    CavityDesc d = make_desc(c, 0);
    if (on_device) {
        for (int q = 0; q < 6; ++q)
            CK(c, launch_pack(c->storage, d, 0, q, f[q], q >= 3 ? c->face[q - 3] : nullptr, c->stream));
    } else {
        // host fields: field q is copied into staging buffer q & 1 on the copy stream while the
        // previous field is packed on the context's stream (the copy waits until buffer q & 1 is free)
        if (int rc = ensure_stage2(c)) return rc;
        CK(c, cudaEventRecord(c->packed[0], c->stream));   // orders the copies after earlier work
        CK(c, cudaEventRecord(c->packed[1], c->stream));
        for (int q = 0; q < 6; ++q) {
            const int b = q & 1;
            float *stage = b ? c->d_stage2 : c->d_stage;
            CK(c, cudaStreamWaitEvent(c->copy_stream, c->packed[b], 0));
            CK(c, cudaMemcpyAsync(stage, f[q], n * 4, cudaMemcpyHostToDevice, c->copy_stream));
            CK(c, cudaEventRecord(c->staged[b], c->copy_stream));
            CK(c, cudaStreamWaitEvent(c->stream, c->staged[b], 0));
            CK(c, launch_pack(c->storage, d, 0, q, stage, q >= 3 ? c->face[q - 3] : nullptr, c->stream));
            CK(c, cudaEventRecord(c->packed[b], c->stream));
        }
    }
    if (c->d_xclock) CK(c, cudaMemsetAsync(c->d_xclock, 0, sizeof(long long), c->stream));
    if (c->d_probe_buf)
        CK(c, cudaMemsetAsync(c->d_probe_buf, 0, sizeof(float) * (size_t)c->nprobe * c->probe_cap, c->stream));
    c->probe_start = 0;
    CK(c, cudaStreamSynchronize(c->stream));
    c->cur = 0;
    c->steps = 0;
    c->has_fields = true;
    return check_status(c, c->d_status, c->stream);
}

int fdtd_prefetch_fields(fdtd_ctx *c, const float *const f[6]) {
    NvtxRange nvtx_range("fdtd_prefetch_fields");
    if (!c || !f) return fail(c, FDTD_ERR_ARG, "NULL argument");
    for (int q = 0; q < 6; ++q)
        if (!f[q]) return fail(c, FDTD_ERR_ARG, "field %d is NULL", q);
    if (c->prefetch_pending) return fail(c, FDTD_ERR_STATE, "a prefetch is pending: load it first");
    if (int rc = ensure_stage2(c)) return rc;   // the copy stream
    const size_t n = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
    if (!c->d_prefetch) {
        CK(c, dmalloc(c, (void **)&c->d_prefetch, 6 * n * sizeof(float)));
        CK(c, cudaEventCreateWithFlags(&c->prefetched, cudaEventDisableTiming));
        CK(c, cudaEventCreateWithFlags(&c->prefetch_free, cudaEventDisableTiming));
        CK(c, cudaEventRecord(c->prefetch_free, c->stream));   // after the allocation on the context stream
    }
    // the previous prefetch's arrays must have been packed before they are overwritten
    CK(c, cudaStreamWaitEvent(c->copy_stream, c->prefetch_free, 0));
    for (int q = 0; q < 6; ++q)
        CK(c, cudaMemcpyAsync(c->d_prefetch + q * n, f[q], n * sizeof(float), cudaMemcpyHostToDevice,
                              c->copy_stream));
    CK(c, cudaEventRecord(c->prefetched, c->copy_stream));
    c->prefetch_pending = true;
    return FDTD_OK;
}

int fdtd_set_fields_prefetched(fdtd_ctx *c) {
    NvtxRange nvtx_range("fdtd_set_fields_prefetched");
    if (!c) return FDTD_ERR_ARG;
    if (!c->prefetch_pending) return fail(c, FDTD_ERR_STATE, "no prefetch pending");
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member; remove it first");
    CK(c, cudaStreamWaitEvent(c->stream, c->prefetched, 0));
    const size_t n = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
    const float *src[6];
    for (int q = 0; q < 6; ++q) src[q] = c->d_prefetch + q * n;
    c->prefetch_pending = false;
    const int rc = fdtd_set_fields(c, src, 1);
    CK(c, cudaEventRecord(c->prefetch_free, c->stream));
    return rc;
}

int fdtd_get_fields(fdtd_ctx *c, float *const f[6], int on_device) {
    NvtxRange nvtx_range("fdtd_get_fields");
    if (!c || !f) return fail(c, FDTD_ERR_ARG, "NULL argument");
    for (int q = 0; q < 6; ++q)
        if (!f[q]) return fail(c, FDTD_ERR_ARG, "field %d is NULL", q);
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member; remove it first");
    const size_t n = (size_t)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
    if (!on_device)
        if (int rc = ensure_stage(c)) return rc;
    CavityDesc d = make_desc(c, 0);
    for (int q = 0; q < 6; ++q) {
        float *dst = on_device ? f[q] : c->d_stage;
        CK(c, launch_unpack(c->storage, d, c->cur, q, dst, c->stream));
        if (!on_device) CK(c, cudaMemcpyAsync(f[q], c->d_stage, n * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return check_status(c, c->d_status, c->stream);
}

int fdtd_step(fdtd_ctx *c, int nsteps) {
    NvtxRange nvtx_range("fdtd_step");
    if (!c) return FDTD_ERR_ARG;
    if (nsteps < 0) return fail(c, FDTD_ERR_ARG, "nsteps < 0");
    if (!c->has_fields) return fail(c, FDTD_ERR_STATE, "fdtd_set_fields has not been called");
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member; step the batch");
    if (nsteps == 0) return FDTD_OK;
    const bool fused = use_fused(c);
    const bool extras = extras_on(c);
    // currents enter between the E update of one step and the H update of the next: one step per launch
    const bool temporal = use_temporal(c) && !extras;
    const int k1 = one_step_kind(c);
    if (fused)
        if (int rc = build_tiles(c, k1)) return rc;
    if (temporal)
        if (int rc = build_tiles(c, 1)) return rc;
    // one launch from copy `parity` (fused kernels write copy parity ^ 1; the unfused one works in
    // place on copy cur), then the point currents and probes of that step
    auto step_launch = [&](int parity, int inj, int kind) -> int {
        if (int rc = launch_one(c, parity, inj, kind)) return rc;
        return extras ? launch_extras_after(c, fused ? parity ^ 1 : c->cur) : FDTD_OK;
    };
    int left = nsteps;
    if (c->inject_us > 0 && fused) {
        const int inj = c->inject_us;
        c->inject_us = 0;
        if (int rc = step_launch(c->cur, inj, k1)) return rc;
        c->cur ^= 1;
        ++c->steps;
        --left;
    }
    // kind 1 advances two steps per launch; either kind reads copy cur and writes copy 1 - cur.
    // An odd remainder takes one launch of the one-step kernel at the end.
    const int kind = temporal ? 1 : k1;
    const int per = temporal ? 2 : 1;
    const int K = 16;   // steps per graph
    if (c->tuning.use_graph && fused && c->stream != nullptr && left >= K) {
        GraphKey key{K, c->cur, kind + (extras ? 4 : 0)};
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            cudaGraph_t g;
            CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            int rc = FDTD_OK;
            for (int s = 0; s < K / per && !rc; ++s) rc = step_launch(c->cur ^ (s & 1), 0, kind);
            cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
            if (rc) return rc;
            CK(c, ee);
            cudaGraphExec_t ex;
            CK(c, cudaGraphInstantiate(&ex, g, 0));
            cudaGraphDestroy(g);
            it = c->graphs.emplace(key, ex).first;
        }
        while (left >= K) {
            CK(c, cudaGraphLaunch(it->second, c->stream));
            left -= K;
            c->steps += K;   // an even number of launches: parity unchanged
        }
    }
    if (temporal)
        for (; left >= 2; left -= 2) {
            if (int rc = step_launch(c->cur, 0, 1)) return rc;
            c->cur ^= 1;
            c->steps += 2;
        }
    for (; left > 0; --left) {
        if (int rc = step_launch(c->cur, 0, k1)) return rc;
        if (fused) c->cur ^= 1;
        ++c->steps;
    }
    return FDTD_OK;
}

// ---------------------------------------------------------------------------------------------
// Point currents and probes.
static int free_extras(fdtd_ctx *c, bool sources, bool probes) {
    CK(c, cudaStreamSynchronize(c->stream));   // no launch may still read the old arrays
    drop_graphs(c->graphs);                   // graphs hold (or lack) the extras launch
    if (sources) {
        for (void *p : {(void *)c->d_src_comp, (void *)c->d_src_off, (void *)c->d_wave}) pool_free(p, c->stream);
        c->d_src_comp = nullptr;
        c->d_src_off = nullptr;
        c->d_wave = nullptr;
        c->nsrc = c->wave_len = 0;
    }
    if (probes) {
        for (void *p : {(void *)c->d_probe_comp, (void *)c->d_probe_off, (void *)c->d_probe_buf})
            pool_free(p, c->stream);
        c->d_probe_comp = nullptr;
        c->d_probe_off = nullptr;
        c->d_probe_buf = nullptr;
        c->nprobe = c->probe_cap = 0;
    }
    return FDTD_OK;
}

// The device step clock, started at the context's step count when the first current or probe is set.
static int ensure_xclock(fdtd_ctx *c) {
    if (c->d_xclock) return FDTD_OK;
    CK(c, pool_alloc((void **)&c->d_xclock, sizeof(long long), c->stream));
    const long long n = c->steps;
    CK(c, cudaMemcpyAsync(c->d_xclock, &n, sizeof n, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FDTD_OK;
}

static int upload(fdtd_ctx *c, void **dst, const void *src, size_t bytes) {
    CK(c, pool_alloc(dst, bytes, c->stream));
    CK(c, cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return FDTD_OK;
}

int fdtd_set_sources(fdtd_ctx *c, int nsrc, const int *comp, const int *ijk, const float *wave, int wave_len) {
    if (!c) return FDTD_ERR_ARG;
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member; remove it first");
    if (nsrc < 0 || (nsrc > 0 && (!comp || !ijk || !wave || wave_len < 1)))
        return fail(c, FDTD_ERR_ARG, "bad source arguments");
    std::vector<long long> off(nsrc);
    for (int s = 0; s < nsrc; ++s) {
        const int q = comp[s], i = ijk[3 * s], j = ijk[3 * s + 1], k = ijk[3 * s + 2];
        // an E position inside the cavity and not tangential to a face (those stay 0: PEC)
        const bool ok = (q == 0 && i >= 0 && i < c->nx && j >= 1 && j < c->ny && k >= 1 && k < c->nz) ||
                        (q == 1 && i >= 1 && i < c->nx && j >= 0 && j < c->ny && k >= 1 && k < c->nz) ||
                        (q == 2 && i >= 1 && i < c->nx && j >= 1 && j < c->ny && k >= 0 && k < c->nz);
        if (!ok) return fail(c, FDTD_ERR_ARG, "source %d: component %d at (%d, %d, %d) is not an interior E position",
                             s, q, i, j, k);
        off[s] = (long long)k * c->pitch * c->ny + (long long)j * c->pitch + i;
    }
    if (int rc = free_extras(c, true, false)) return rc;
    if (nsrc == 0) return FDTD_OK;
    if (int rc = upload(c, (void **)&c->d_src_comp, comp, sizeof(int) * nsrc)) return rc;
    if (int rc = upload(c, (void **)&c->d_src_off, off.data(), sizeof(long long) * nsrc)) return rc;
    if (int rc = upload(c, (void **)&c->d_wave, wave, sizeof(float) * (size_t)nsrc * wave_len)) return rc;
    CK(c, cudaStreamSynchronize(c->stream));
    c->nsrc = nsrc;
    c->wave_len = wave_len;
    return ensure_xclock(c);
}

int fdtd_set_probes(fdtd_ctx *c, int nprobe, const int *comp, const int *ijk, int capacity) {
    if (!c) return FDTD_ERR_ARG;
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member; remove it first");
    if (nprobe < 0 || (nprobe > 0 && (!comp || !ijk || capacity < 1)))
        return fail(c, FDTD_ERR_ARG, "bad probe arguments");
    std::vector<long long> off(nprobe);
    for (int p = 0; p < nprobe; ++p) {
        const int q = comp[p], i = ijk[3 * p], j = ijk[3 * p + 1], k = ijk[3 * p + 2];
        if (q < 0 || q > 5 || i < 0 || i >= c->nx || j < 0 || j >= c->ny || k < 0 || k >= c->nz)
            return fail(c, FDTD_ERR_ARG, "probe %d: component %d at (%d, %d, %d) is outside [0,nx)x[0,ny)x[0,nz)",
                        p, q, i, j, k);
        off[p] = (long long)k * c->pitch * c->ny + (long long)j * c->pitch + i;
    }
    if (int rc = free_extras(c, false, true)) return rc;
    if (nprobe == 0) return FDTD_OK;
    if (int rc = upload(c, (void **)&c->d_probe_comp, comp, sizeof(int) * nprobe)) return rc;
    if (int rc = upload(c, (void **)&c->d_probe_off, off.data(), sizeof(long long) * nprobe)) return rc;
    CK(c, pool_alloc((void **)&c->d_probe_buf, sizeof(float) * (size_t)nprobe * capacity, c->stream));
    CK(c, cudaMemsetAsync(c->d_probe_buf, 0, sizeof(float) * (size_t)nprobe * capacity, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->nprobe = nprobe;
    c->probe_cap = capacity;
    c->probe_start = c->steps;
    return ensure_xclock(c);
}

int fdtd_get_probes(fdtd_ctx *c, float *out, int *nrecorded) {
    if (!c || !out || !nrecorded) return fail(c, FDTD_ERR_ARG, "NULL argument");
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member; remove it first");
    if (c->nprobe == 0) return fail(c, FDTD_ERR_STATE, "no probes are set");
    long long n = 0;
    CK(c, cudaMemcpyAsync(&n, c->d_xclock, sizeof n, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(out, c->d_probe_buf, sizeof(float) * (size_t)c->nprobe * c->probe_cap,
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *nrecorded = (int)std::max<long long>(0, std::min<long long>(c->probe_cap, n - c->probe_start));
    return check_status(c, c->d_status, c->stream);
}

int fdtd_sync(fdtd_ctx *c) {
    if (!c) return FDTD_ERR_ARG;
    CK(c, cudaStreamSynchronize(c->stream));
    return check_status(c, c->d_status, c->stream);
}

static int run_reductions(fdtd_ctx *c, int what, double out[3]) {
    if (!c->has_fields) return fail(c, FDTD_ERR_STATE, "fdtd_set_fields has not been called");
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member; remove it first");
    CK(c, launch_reductions(c->storage, make_desc(c, 0), c->cur, what, c->d_partial, reduction_blocks(), c->d_out,
                            c->stream, c->order));
    CK(c, cudaMemcpyAsync(out, c->d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return check_status(c, c->d_status, c->stream);
}

int fdtd_energy(fdtd_ctx *c, double *W) {
    NvtxRange nvtx_range("fdtd_energy");
    if (!c || !W) return fail(c, FDTD_ERR_ARG, "NULL argument");
    double o[3];
    if (int rc = run_reductions(c, 0, o)) return rc;
    *W = 0.5 * (c->dt / c->dx) * o[0];
    return FDTD_OK;
}

int fdtd_divergence(fdtd_ctx *c, double *de, double *dh) {
    NvtxRange nvtx_range("fdtd_divergence");
    if (!c || !de || !dh) return fail(c, FDTD_ERR_ARG, "NULL argument");
    double o[3];
    if (int rc = run_reductions(c, 1, o)) return rc;
    *de = std::sqrt(o[1]);
    *dh = std::sqrt(o[2]);
    return FDTD_OK;
}

int fdtd_debug_fail_alloc(int after) {
    g_fail_alloc_in.store(after < 0 ? -1 : after);
    return FDTD_OK;
}

int fdtd_debug_tile_plan(long long cols, int nz, int ctas, int prologue, int zchunk, int *chunks, int max_chunks,
                         int *nchunks, long long *makespan, int *cta_of_tile) {
    if (cols < 1 || nz < 1 || ctas < 1 || prologue < 0 || zchunk < 0 || !chunks || !nchunks || !makespan)
        return FDTD_ERR_ARG;
    // the same sequence as build_tiles with one CTA per SM: plan for G CTAs, list chunk-major, assign greedily
    const int G = (int)std::min<long long>(ctas, cols * nz);
    const std::vector<int> plan = plan_chunks(cols, nz, G, prologue, zchunk);
    if ((int)plan.size() > max_chunks) return FDTD_ERR_ARG;
    const long long ntiles = cols * (long long)plan.size();
    if (cta_of_tile && ntiles > (1ll << 26)) return FDTD_ERR_ARG;
    for (size_t q = 0; q < plan.size(); ++q) chunks[q] = plan[q];
    *nchunks = (int)plan.size();
    *makespan = simulate_plan(plan, cols, G, prologue);
    if (cta_of_tile) {
        std::vector<TileRec> listed;
        listed.reserve((size_t)ntiles);
        int z0 = 0;
        for (int len : plan) {
            for (long long col = 0; col < cols; ++col) {
                TileRec t{};
                t.x0 = (int)listed.size();   // the listing index, to map the regrouped records back
                t.kz0 = z0;
                t.kz1 = z0 + len;
                listed.push_back(t);
            }
            z0 += len;
        }
        std::vector<int> first;
        const int grid = (int)std::min<long long>(ntiles, G);
        const std::vector<TileRec> v = assign_tiles(listed, grid, prologue, first);
        for (int b = 0; b < grid; ++b)
            for (int q = first[b]; q < first[b + 1]; ++q) cta_of_tile[v[q].x0] = b;
    }
    return FDTD_OK;
}

int fdtd_debug_inject_timeout(fdtd_ctx *c, int limit_us) {
    if (!c) return FDTD_ERR_ARG;
    if (limit_us < 1 || limit_us > 1000000) return fail(c, FDTD_ERR_ARG, "limit_us must be in [1, 1e6]");
    if (!use_fused(c)) return fail(c, FDTD_ERR_STATE, "timeout injection needs the fused kernel");
    c->inject_us = limit_us;
    return FDTD_OK;
}

// ------------------------------------------------------------------ batches

int fdtd_batch_create(fdtd_batch **out, int storage, void *cuda_stream) {
    if (!out) return FDTD_ERR_ARG;
    *out = nullptr;
    if (storage < FDTD_F32 || storage > FDTD_BF16) return FDTD_ERR_ARG;
    fdtd_batch *b = new fdtd_batch();
    b->storage = storage;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    bool ok = pool_alloc((void **)&b->d_status, sizeof(int), b->stream) == cudaSuccess &&
              pool_alloc((void **)&b->d_step, sizeof(long long), b->stream) == cudaSuccess &&
              cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream) == cudaSuccess &&
              cudaMemsetAsync(b->d_step, 0, sizeof(long long), b->stream) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done_ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamSynchronize(b->stream) == cudaSuccess;
    if (!ok) {
        pool_free(b->d_status, b->stream);
        pool_free(b->d_step, b->stream);
        if (b->done_ev) cudaEventDestroy(b->done_ev);
        delete b;
        return FDTD_ERR_OOM;
    }
    *out = b;
    return FDTD_OK;
}

int fdtd_batch_size(const fdtd_batch *b) { return b ? (int)b->members.size() : -1; }
const char *fdtd_batch_last_error(const fdtd_batch *b) { return b ? b->err.c_str() : ""; }
long long fdtd_batch_steps_done(const fdtd_batch *b) { return b ? b->step : -1; }

static fdtd_batch::Member *find_member(fdtd_batch *b, fdtd_ctx *c, size_t *idx = nullptr) {
    for (size_t n = 0; n < b->members.size(); ++n)
        if (b->members[n].c == c) {
            if (idx) *idx = n;
            return &b->members[n];
        }
    return nullptr;
}

int fdtd_batch_add(fdtd_batch *b, fdtd_ctx *c) {
    if (!b || !c) return bfail(b, FDTD_ERR_ARG, "NULL argument");
    if (c->batch) return bfail(b, FDTD_ERR_STATE, "context already belongs to a batch");
    if (!c->has_fields) return bfail(b, FDTD_ERR_STATE, "context has no fields yet");
    if (c->storage != b->storage) return bfail(b, FDTD_ERR_ARG, "storage mismatch");
    if (c->coef_mode == COEF_FULL) return bfail(b, FDTD_ERR_ARG, "per-position coefficient arrays are not batched");
    if (extras_on(c)) return bfail(b, FDTD_ERR_ARG, "contexts with currents or probes are not batched");
    if (c->order != 2) return bfail(b, FDTD_ERR_ARG, "fourth-order contexts are not batched");
    // the member's pending work (set_fields) happened-before: its stream was synchronised by that call
    b->members.push_back({c, c->cur, b->step, b->launches, LLONG_MAX, c->steps, 0});
    c->batch = b;
    b->dirty = true;
    return FDTD_OK;
}

int fdtd_batch_set_steps(fdtd_batch *b, fdtd_ctx *c, long long nsteps) {
    if (!b || !c || nsteps < 0) return bfail(b, FDTD_ERR_ARG, "bad argument");
    fdtd_batch::Member *mb = find_member(b, c);
    if (!mb) return bfail(b, FDTD_ERR_ARG, "context is not a member");
    mb->stop = b->step + nsteps;
    b->dirty = true;
    return FDTD_OK;
}

int fdtd_batch_remove(fdtd_batch *b, fdtd_ctx *c) {
    if (!b || !c) return bfail(b, FDTD_ERR_ARG, "NULL argument");
    size_t n = 0;
    fdtd_batch::Member *mb = find_member(b, c, &n);
    if (!mb) return bfail(b, FDTD_ERR_ARG, "context is not a member");
    const long long last = std::min(b->step, mb->stop);   // clock after the member's last step
    const long long taken = last - mb->join;
    c->cur = mb->cur0 ^ (int)(mb->nlaunch & 1);
    c->steps = mb->steps0 + taken;
    c->batch = nullptr;
    // later work on the member's own stream (read-back, destroy) waits for the batch launches that
    // touched it: those up to the first completion mark at or past its last step
    if (taken > 0 || mb->nlaunch > 0) {
        cudaEvent_t ev = nullptr;
        for (const auto &mk : b->marks)
            if (mk.first >= last) {
                ev = mk.second;
                break;
            }
        if (!ev) {   // no mark covers it yet (not possible after fdtd_batch_step): wait for everything
            if (cudaEventRecord(b->done_ev, b->stream) != cudaSuccess)
                return bfail(b, FDTD_ERR_CUDA, "ordering the member's stream after the batch failed");
            ev = b->done_ev;
        }
        if (cudaStreamWaitEvent(c->stream, ev, 0) != cudaSuccess)
            return bfail(b, FDTD_ERR_CUDA, "ordering the member's stream after the batch failed");
    }
    b->members.erase(b->members.begin() + n);
    b->dirty = true;
    return FDTD_OK;
}

int fdtd_batch_set_tuning(fdtd_batch *b, const fdtd_tuning *t) {
    if (!b) return FDTD_ERR_ARG;
    fdtd_tuning n{};
    if (t) n = *t;
    if (n.kernel == FDTD_KERNEL_SIMPLE || n.kernel < 0 || n.kernel > FDTD_KERNEL_TEMPORAL)
        return bfail(b, FDTD_ERR_ARG, "batches use the fused kernels (FUSED or TEMPORAL)");
    const bool ty_one = n.tile_y == 4 || n.tile_y == 8 || n.tile_y == 16,
               ty_two = n.tile_y == 8 || n.tile_y == 12 || n.tile_y == 16;
    if (n.tile_y && !(n.kernel == FDTD_KERNEL_TEMPORAL ? ty_two
                      : n.kernel == FDTD_KERNEL_AUTO   ? (ty_one || ty_two)
                                                       : ty_one))
        return bfail(b, FDTD_ERR_ARG, "bad tile_y");
    if (n.stages && (n.stages < 3 || n.stages > 8)) return bfail(b, FDTD_ERR_ARG, "bad stages");
    b->tuning = n;
    b->dirty = true;
    return FDTD_OK;
}

static void batch_retire_graphs(fdtd_batch *b) {
    for (auto &kv : b->graphs) b->retired_graphs.push_back(kv.second);
    b->graphs.clear();
}

static void batch_free_retired_graphs(fdtd_batch *b) {   // call only when the batch stream is idle
    for (cudaGraphExec_t g : b->retired_graphs) cudaGraphExecDestroy(g);
    b->retired_graphs.clear();
}

static int batch_kind(const fdtd_batch *b) {
    return b->tuning.kernel == FDTD_KERNEL_TEMPORAL || b->tuning.kernel == FDTD_KERNEL_AUTO ? 1 : 0;
}

// Rebuild the packed tile list (asynchronously on the batch stream: the upload runs after the
// launches already enqueued, and the old buffer is released in stream order).
static int batch_rebuild(fdtd_batch *b) {
    if (!b->dirty) return FDTD_OK;
    batch_retire_graphs(b);
    const int kind = batch_kind(b);
    Shape s = resolve_shape(b->storage, b->tuning, kind);
    const int box_y = s.tile_y + (kind == 0 ? 2 : 4);
    const int G = num_sms() * s.ctas_per_sm;
    std::vector<TileRec> tiles;
    long long total_cols_planes = 0;
    for (auto &mb : b->members)
        if (mb.stop > b->step && mb.c->maps_by[kind] != 0 && mb.c->maps_by[kind] != box_y) {
            cudaStreamSynchronize(b->stream);   // launches in flight may still read the old maps
            break;
        }
    const int tw = kind == 0 ? kTileX : fused2_tile_w(b->storage);
    for (auto &mb : b->members) {
        if (mb.stop <= b->step) continue;   // finished members carry no tiles
        fdtd_ctx *c = mb.c;
        if (int rc = encode_maps(c, kind, box_y)) return bfail(b, rc, "member: %s", c->err.c_str());
        total_cols_planes += (long long)((c->nx + tw - 1) / tw) * ((c->ny + s.tile_y - 1) / s.tile_y) * c->nz;
    }
    // one z-length for all members so tiles carry similar work; about 8 tiles per CTA
    const int zlen = b->tuning.zchunk > 0 ? b->tuning.zchunk
                                          : (int)std::max<long long>(8, total_cols_planes / std::max(1, 8 * G));
    for (auto &mb : b->members) {
        if (mb.stop <= b->step) continue;
        const size_t first = tiles.size();
        append_tiles(tiles, mb.c, mb.cur0 ^ (int)(mb.join_launch & 1), s.tile_y, std::min(zlen, mb.c->nz), kind);
        for (size_t q = first; q < tiles.size(); ++q) tiles[q].stop = mb.stop;
    }
    // longest tiles first, then round-robin over the persistent CTAs
    std::stable_sort(tiles.begin(), tiles.end(),
                     [](const TileRec &a, const TileRec &c) { return (a.kz1 - a.kz0) > (c.kz1 - c.kz0); });
    if ((int)tiles.size() > b->tiles_cap) {
        pool_free(b->d_tiles, b->stream);
        b->d_tiles = nullptr;
        b->tiles_cap = std::max<int>((int)tiles.size(), 2 * b->tiles_cap);
        if (pool_alloc((void **)&b->d_tiles, sizeof(TileRec) * b->tiles_cap, b->stream) != cudaSuccess)
            return bfail(b, FDTD_ERR_OOM, "tile list alloc");
    }
    if (!tiles.empty() && cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(TileRec) * tiles.size(),
                                          cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return bfail(b, FDTD_ERR_CUDA, "tile list upload");
    b->ntiles = (int)tiles.size();
    b->grid = std::min(b->ntiles, G);
    b->dirty = false;
    return FDTD_OK;
}

// One launch advancing the batch clock by nsteps (1, or 2 with the two-step kernel), then the clock.
static int batch_launch(fdtd_batch *b, int parity, int nsteps) {
    const int kind = batch_kind(b);
    Shape s = resolve_shape(b->storage, b->tuning, kind);
    FusedLaunch L{};
    L.recs = b->d_tiles;
    L.step = b->d_step;
    L.ntiles = b->ntiles;
    L.parity = parity;
    L.status = b->d_status;
    L.tile_y = s.tile_y;
    L.stages = s.stages;
    L.grid = b->grid;
    L.launch_steps = nsteps;
    cudaError_t e = kind == 0 ? launch_fused_step(b->storage, L, b->stream) : launch_fused2_step(b->storage, L, b->stream);
    if (e == cudaSuccess) e = launch_step_counter(b->d_step, nsteps, b->stream);
    if (e != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
    return FDTD_OK;
}

// Host bookkeeping of one launch that starts at the current clock: members with steps left take part.
static void batch_account(fdtd_batch *b, int nsteps) {
    for (auto &mb : b->members)
        if (mb.stop > b->step) ++mb.nlaunch;
    b->step += nsteps;
    ++b->launches;
}

int fdtd_batch_step(fdtd_batch *b, int nsteps) {
    NvtxRange nvtx_range("fdtd_batch_step");
    if (!b || nsteps < 0) return bfail(b, FDTD_ERR_ARG, "bad argument");
    if (b->members.empty() || nsteps == 0) return FDTD_OK;
    if (int rc = batch_rebuild(b)) return rc;
    const int kind = batch_kind(b);
    const int per = kind == 0 ? 1 : 2;   // steps per launch
    int left = nsteps;
    const int K = 16;                    // steps per graph (an even number of launches: parity unchanged)
    if (b->tuning.use_graph && b->stream != nullptr && left >= K) {
        const int par = (int)(b->launches & 1);
        GraphKey key{K, par, kind};
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t g;
            if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return bfail(b, FDTD_ERR_CUDA, "capture");
            int rc = FDTD_OK;
            for (int q = 0; q < K / per && !rc; ++q) rc = batch_launch(b, par ^ (q & 1), per);
            cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
            if (rc) return rc;
            if (ee != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "end capture: %s", cudaGetErrorString(ee));
            cudaGraphExec_t ex;
            if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
                cudaGraphDestroy(g);
                return bfail(b, FDTD_ERR_CUDA, "instantiate");
            }
            cudaGraphDestroy(g);
            it = b->graphs.emplace(key, ex).first;
        }
        while (left >= K) {
            if (cudaGraphLaunch(it->second, b->stream) != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "graph launch");
            for (int q = 0; q < K / per; ++q) batch_account(b, per);
            left -= K;
        }
    }
    while (left > 0) {
        const int n = std::min(per, left);   // a two-step batch ends an odd count with a level-1 launch
        if (int rc = batch_launch(b, (int)(b->launches & 1), n)) return rc;
        batch_account(b, n);
        left -= n;
    }
    // completion mark at the new clock; marks whose work has finished are recycled (the newest stays)
    while (b->marks.size() > 1 && cudaEventQuery(b->marks.front().second) == cudaSuccess) {
        b->free_marks.push_back(b->marks.front().second);
        b->marks.pop_front();
    }
    cudaEvent_t ev = nullptr;
    if (!b->free_marks.empty()) {
        ev = b->free_marks.back();
        b->free_marks.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        return bfail(b, FDTD_ERR_CUDA, "event create");
    }
    if (cudaEventRecord(ev, b->stream) != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "event record");
    b->marks.emplace_back(b->step, ev);
    return FDTD_OK;
}

int fdtd_batch_autotune(fdtd_batch *b, int trial_steps, fdtd_tuning *out, double *ms_per_step) {
    NvtxRange nvtx_range("fdtd_batch_autotune");
    if (!b) return FDTD_ERR_ARG;
    if (b->members.empty()) return bfail(b, FDTD_ERR_STATE, "autotune: the batch has no members");
    const int n = trial_length(trial_steps);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "sync");
    // each member's current copy, set aside; the clock and launch counts are restored afterwards
    struct Saved {
        char *snap;
        size_t bytes;
        int copy;
        long long nlaunch;
    };
    std::vector<Saved> saved;
    int rc = FDTD_OK;
    for (auto &mb : b->members) {
        fdtd_ctx *c = mb.c;
        Saved sv{nullptr, (size_t)c->pitch * c->ny * c->nz * esize(c->storage), mb.cur0 ^ (int)(mb.nlaunch & 1),
                 mb.nlaunch};
        if (pool_alloc((void **)&sv.snap, 6 * sv.bytes, b->stream) != cudaSuccess) {
            rc = bfail(b, FDTD_ERR_OOM, "autotune: no room for a copy of the members' fields");
            break;
        }
        for (int f = 0; f < 6; ++f)
            cudaMemcpyAsync(sv.snap + f * sv.bytes, c->fields[sv.copy][f], sv.bytes, cudaMemcpyDeviceToDevice,
                            b->stream);
        saved.push_back(sv);
    }
    const long long step0 = b->step, launches0 = b->launches;
    const fdtd_tuning t0 = b->tuning;
    fdtd_tuning best = t0;
    double best_ms = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = bfail(b, FDTD_ERR_CUDA, "event create");
    if (!rc)
        for (const fdtd_tuning &t : tune_candidates(true)) {
            if ((rc = fdtd_batch_set_tuning(b, &t)) != FDTD_OK) break;
            if ((rc = fdtd_batch_step(b, n)) != FDTD_OK) break;
            cudaEventRecord(e0, b->stream);
            if ((rc = fdtd_batch_step(b, n)) != FDTD_OK) break;
            cudaEventRecord(e1, b->stream);
            if ((rc = fdtd_batch_sync(b)) != FDTD_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best_ms < 0 || ms / n < best_ms) {
                best_ms = ms / n;
                best = t;
            }
        }
    cudaStreamSynchronize(b->stream);
    for (size_t q = 0; q < saved.size(); ++q) {
        fdtd_batch::Member &mb = b->members[q];
        for (int f = 0; f < 6; ++f)
            cudaMemcpyAsync(mb.c->fields[saved[q].copy][f], saved[q].snap + f * saved[q].bytes, saved[q].bytes,
                            cudaMemcpyDeviceToDevice, b->stream);
        pool_free(saved[q].snap, b->stream);
        mb.nlaunch = saved[q].nlaunch;
    }
    b->step = step0;
    b->launches = launches0;
    cudaMemcpyAsync(b->d_step, &step0, sizeof(long long), cudaMemcpyHostToDevice, b->stream);
    cudaStreamSynchronize(b->stream);   // step0 is read by the copy above before it goes out of scope
    for (auto &mk : b->marks) b->free_marks.push_back(mk.second);   // their clocks ran ahead of the restored one
    b->marks.clear();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->dirty = true;
    if (rc != FDTD_OK) {
        b->tuning = t0;
        return rc;
    }
    if (int r2 = fdtd_batch_set_tuning(b, &best)) return r2;
    if (out) *out = best;
    if (ms_per_step) *ms_per_step = best_ms;
    return FDTD_OK;
}

// ---------------------------------------------------------------------------------------------
// Online re-tuning: a size-bucket model of batch tunings.  A bucket is (storage, floor(log2 of the
// running members' total cells)); the first batch seen in a bucket is timed by fdtd_batch_autotune,
// later ones take the bucket's choice without trials.
namespace {

std::mutex g_btune_mu;
std::map<std::pair<int, int>, std::pair<fdtd_tuning, double>> g_btune_cache;

int floor_log2(long long v) {
    int r = 0;
    while (v > 1) {
        v >>= 1;
        ++r;
    }
    return r;
}

bool same_tuning(const fdtd_tuning &a, const fdtd_tuning &b) {
    return a.kernel == b.kernel && a.tile_y == b.tile_y && a.zchunk == b.zchunk && a.ctas_per_sm == b.ctas_per_sm &&
           a.stages == b.stages && a.use_graph == b.use_graph;
}

}  // namespace

int fdtd_batch_retune(fdtd_batch *b, int trial_steps, fdtd_tuning *out, double *ms_per_step, int *timed) {
    if (!b) return FDTD_ERR_ARG;
    if (b->members.empty()) return bfail(b, FDTD_ERR_STATE, "retune: the batch has no members");
    long long cells = 0, running = 0;
    for (const auto &mb : b->members)
        if (mb.stop > b->step) {
            cells += (long long)mb.c->nx * mb.c->ny * mb.c->nz;
            ++running;
        }
    if (running == 0)   // every member has taken its steps: bucket by all of them
        for (const auto &mb : b->members) {
            cells += (long long)mb.c->nx * mb.c->ny * mb.c->nz;
            ++running;
        }
    const auto key = std::make_pair(b->storage, floor_log2(cells));
    fdtd_tuning t{};
    double ms = -1.0;
    bool hit = false;
    {
        std::lock_guard<std::mutex> g(g_btune_mu);
        auto it = g_btune_cache.find(key);
        if (it != g_btune_cache.end()) {
            t = it->second.first;
            ms = it->second.second;
            hit = true;
        }
    }
    if (hit) {
        if (!same_tuning(t, b->tuning))
            if (int rc = fdtd_batch_set_tuning(b, &t)) return rc;
    } else {
        if (int rc = fdtd_batch_autotune(b, trial_steps, &t, &ms)) return rc;
        std::lock_guard<std::mutex> g(g_btune_mu);
        g_btune_cache[key] = {t, ms};
    }
    if (out) *out = t;
    if (ms_per_step) *ms_per_step = ms;
    if (timed) *timed = hit ? 0 : 1;
    return FDTD_OK;
}

int fdtd_batch_sync(fdtd_batch *b) {
    if (!b) return FDTD_ERR_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "sync");
    batch_free_retired_graphs(b);
    int h = 0;
    if (cudaMemcpy(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return bfail(b, FDTD_ERR_CUDA, "status read");
    if (h) {
        cudaMemset(b->d_status, 0, sizeof(int));
        return bfail(b, (h & STATUS_TIMEOUT) ? FDTD_ERR_TIMEOUT : FDTD_ERR_CUDA, "device status 0x%x", h);
    }
    return FDTD_OK;
}

void fdtd_batch_destroy(fdtd_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    while (!b->members.empty()) fdtd_batch_remove(b, b->members.back().c);
    cudaStreamSynchronize(b->stream);
    batch_retire_graphs(b);
    batch_free_retired_graphs(b);
    pool_free(b->d_tiles, b->stream);
    pool_free(b->d_status, b->stream);
    pool_free(b->d_step, b->stream);
    cudaStreamSynchronize(b->stream);
    cudaEventDestroy(b->done_ev);
    for (auto &mk : b->marks) cudaEventDestroy(mk.second);
    for (cudaEvent_t e : b->free_marks) cudaEventDestroy(e);
    delete b;
}

}  // extern "C"
