// Batches of cavities (continuous batching): the packed tile list over all members, persistent
// launches of the fused kernels with a device step clock, per-member stop clocks, CUDA-graph replay
// and completion marks that let a removed member's stream wait only for the launches that touched it.
#include "api_internal.h"

using namespace fdtd;

extern "C" {

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
    if (c->slab.on) return bfail(b, FDTD_ERR_ARG, "slab contexts are not batched");
    // one spatial order per batch (the first member's; the kernel differs): second and fourth-order
    // members go to batches of their own
    if (!b->members.empty() && c->order != b->order)
        return bfail(b, FDTD_ERR_ARG, "the batch runs order %d; this context has order %d", b->order, c->order);
    if (b->members.empty()) b->order = c->order;
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
    if (n.kernel == FDTD_KERNEL_SIMPLE || n.kernel < 0 || n.kernel > FDTD_KERNEL_TEMPORAL2)
        return bfail(b, FDTD_ERR_ARG, "batches use the fused kernels (FUSED, TEMPORAL or TEMPORAL2)");
    // FUSED: 4, 8 or 16 rows (12 too for fourth-order batches; a one-step second-order batch takes its
    // default for it)
    const bool ty_one = n.tile_y == 4 || n.tile_y == 8 || n.tile_y == 12 || n.tile_y == 16,
               ty_two = n.tile_y == 8 || n.tile_y == 12 || n.tile_y == 16, ty_two2 = n.tile_y == 12 || n.tile_y == 16;
    if (n.tile_y && !(n.kernel == FDTD_KERNEL_TEMPORAL    ? ty_two
                      : n.kernel == FDTD_KERNEL_TEMPORAL2 ? ty_two2
                      : n.kernel == FDTD_KERNEL_AUTO      ? (ty_one || ty_two)
                                                          : ty_one))
        return bfail(b, FDTD_ERR_ARG, "bad tile_y");
    if (n.stages && (n.stages < 3 || n.stages > 8)) return bfail(b, FDTD_ERR_ARG, "bad stages");
    b->tuning = n;
    b->dirty = true;
    return FDTD_OK;
}

static void batch_retire_graphs(fdtd_batch *b) {
    for (auto &kv : b->graphs) b->retired_graphs.emplace_back(b->step, kv.second);
    b->graphs.clear();
}

static void batch_free_retired_graphs(fdtd_batch *b) {   // call only when the batch stream is idle
    for (auto &rg : b->retired_graphs) cudaGraphExecDestroy(rg.second);
    b->retired_graphs.clear();
}

// Destroys the retired graphs whose last launches are done: a graph retired at clock c was last launched
// before the completion mark at clock c was recorded.
static void batch_free_finished_graphs(fdtd_batch *b, long long done_clock) {
    size_t keep = 0;
    for (size_t q = 0; q < b->retired_graphs.size(); ++q) {
        if (b->retired_graphs[q].first <= done_clock)
            cudaGraphExecDestroy(b->retired_graphs[q].second);
        else
            b->retired_graphs[keep++] = b->retired_graphs[q];
    }
    b->retired_graphs.resize(keep);
}

// Tile kind of the batch's launches: 2 (the fused fourth-order kernel) for a fourth-order batch whatever the
// tuning's kernel, else 1 (two steps per launch) or 0 (one step).
static int batch_kind(const fdtd_batch *b) {
    if (b->order == 4) return 2;
    return b->tuning.kernel == FDTD_KERNEL_TEMPORAL || b->tuning.kernel == FDTD_KERNEL_TEMPORAL2 ||
                   b->tuning.kernel == FDTD_KERNEL_AUTO
               ? 1
               : 0;
}

// Rebuild the packed tile list (asynchronously on the batch stream: the upload runs after the
// launches already enqueued, and the old buffer is released in stream order).
static int batch_rebuild(fdtd_batch *b) {
    if (!b->dirty) return FDTD_OK;
    batch_retire_graphs(b);
    const int kind = batch_kind(b);
    Shape s = resolve_shape(b->storage, b->tuning, kind);
    const int box_y = s.tile_y + (kind == 0 ? 2 : kind == 1 ? 4 : 6);
    const int G = num_sms() * s.ctas_per_sm;
    std::vector<TileRec> tiles;
    long long total_cols_planes = 0;
    for (auto &mb : b->members)
        if (mb.stop > b->step && mb.c->maps_by[kind] != 0 && mb.c->maps_by[kind] != box_y) {
            cudaStreamSynchronize(b->stream);   // launches in flight may still read the old maps
            break;
        }
    const int tw = kind == 1 ? fused2_tile_w(b->storage) : kTileX;
    long long total_cols = 0;
    bool same_stop = true;   // every running member stops at the same clock (or never)
    long long stop0 = -1;
    for (auto &mb : b->members) {
        if (mb.stop <= b->step) continue;   // finished members carry no tiles
        fdtd_ctx *c = mb.c;
        if (int rc = encode_maps(c, kind, box_y)) return bfail(b, rc, "member: %s", c->err.c_str());
        const long long cols = (long long)((c->nx + tw - 1) / tw) * ((c->ny + s.tile_y - 1) / s.tile_y);
        total_cols += cols;
        total_cols_planes += cols * c->nz;
        if (stop0 < 0) stop0 = mb.stop;
        same_stop = same_stop && mb.stop == stop0;
    }
    // tiles assigned to the CTAs on the host (below) when every tile takes part in every launch
    const bool balanced = s.ctas_per_sm == 1 && same_stop;
    // One z-length for all members so tiles carry similar work: about 8 tiles per CTA; with balanced ranges
    // and at least 4 tile columns per CTA, whole members (fewer tile prologues; 0.9 % faster on 256 members
    // of sides 16..96)
    const int zlen = b->tuning.zchunk > 0              ? b->tuning.zchunk
                     : (balanced && total_cols >= 4LL * G) ? INT_MAX
                                                         : (int)std::max<long long>(8, total_cols_planes / std::max(1, 8 * G));
    for (auto &mb : b->members) {
        if (mb.stop <= b->step) continue;
        const size_t first = tiles.size();
        append_tiles(tiles, mb.c, mb.cur0 ^ (int)(mb.join_launch & 1), s.tile_y, std::min(zlen, mb.c->nz), kind);
        for (size_t q = first; q < tiles.size(); ++q) tiles[q].stop = mb.stop;
    }
    // Longest tiles first.  When every running member stops at the same clock (or never), every tile takes
    // part in every launch, and with one CTA per SM each tile goes to the CTA that frees first (host-balanced
    // contiguous ranges, as for a single cavity).  Otherwise (members with their own step counts, as in
    // serving) tiles drop out at different clocks and the round-robin deal spreads the holes over the CTAs;
    // co-resident CTAs always take their tiles round-robin.
    std::stable_sort(tiles.begin(), tiles.end(),
                     [](const TileRec &a, const TileRec &c) { return (a.kz1 - a.kz0) > (c.kz1 - c.kz0); });
    const int grid = std::min((int)tiles.size(), G);
    std::vector<int> first;
    if (balanced && !tiles.empty())
        tiles = assign_tiles(tiles, grid, kind == 0 ? 1 : kind == 1 ? 3 : 4, first);
    if ((int)tiles.size() > b->tiles_cap || !b->d_tiles) {
        pool_free(b->d_tiles, b->stream);
        b->d_tiles = nullptr;
        b->tiles_cap = std::max<int>((int)tiles.size(), 2 * b->tiles_cap);
        // room for the records and for the range offsets of up to two CTAs per SM
        const size_t bytes = sizeof(TileRec) * b->tiles_cap + sizeof(int) * (2 * num_sms() + 1);
        if (pool_alloc((void **)&b->d_tiles, bytes, b->stream) != cudaSuccess) return bfail(b, FDTD_ERR_OOM, "tile list alloc");
    }
    // upload through the pinned staging buffer whose previous upload (two rebuilds ago) has finished
    const size_t rec_bytes = sizeof(TileRec) * tiles.size(), first_bytes = sizeof(int) * first.size();
    const int si = b->h_stage_next;
    b->h_stage_next ^= 1;
    if (b->h_stage_ev[si]) {
        if (cudaEventSynchronize(b->h_stage_ev[si]) != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "staging wait");
    } else if (cudaEventCreateWithFlags(&b->h_stage_ev[si], cudaEventDisableTiming) != cudaSuccess) {
        return bfail(b, FDTD_ERR_CUDA, "event create");
    }
    if (b->h_stage_cap[si] < rec_bytes + first_bytes) {
        cudaFreeHost(b->h_stage[si]);
        b->h_stage[si] = nullptr;
        b->h_stage_cap[si] = 0;
        const size_t cap = std::max(rec_bytes + first_bytes, 2 * b->h_stage_cap[si ^ 1]);
        if (cudaMallocHost(&b->h_stage[si], cap) != cudaSuccess) return bfail(b, FDTD_ERR_OOM, "pinned staging alloc");
        b->h_stage_cap[si] = cap;
    }
    char *stage = static_cast<char *>(b->h_stage[si]);
    if (rec_bytes) memcpy(stage, tiles.data(), rec_bytes);
    if (first_bytes) memcpy(stage + rec_bytes, first.data(), first_bytes);
    if (rec_bytes && cudaMemcpyAsync(b->d_tiles, stage, rec_bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
        return bfail(b, FDTD_ERR_CUDA, "tile list upload");
    b->d_first = nullptr;
    if (first_bytes) {
        b->d_first = reinterpret_cast<int *>(b->d_tiles + b->tiles_cap);
        if (cudaMemcpyAsync(b->d_first, stage + rec_bytes, first_bytes, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess)
            return bfail(b, FDTD_ERR_CUDA, "tile range upload");
    }
    if (cudaEventRecord(b->h_stage_ev[si], b->stream) != cudaSuccess) return bfail(b, FDTD_ERR_CUDA, "event record");
    b->ntiles = (int)tiles.size();
    b->grid = grid;
    b->dirty = false;
    return FDTD_OK;
}

// One launch advancing the batch clock by nsteps (1, or 2 with the two-step kernel), then the clock.
static int batch_launch(fdtd_batch *b, int parity, int nsteps) {
    const int kind = batch_kind(b);
    Shape s = resolve_shape(b->storage, b->tuning, kind);
    FusedLaunch L{};
    L.recs = b->d_tiles;
    L.first = b->d_first;
    L.step = b->d_step;
    L.ntiles = b->ntiles;
    L.parity = parity;
    L.status = b->d_status;
    L.tile_y = s.tile_y;
    L.stages = s.stages;
    L.grid = b->grid;
    L.launch_steps = nsteps;
    L.rows_per_warp = s.rows_per_warp;
    cudaError_t e = kind == 0   ? launch_fused_step(b->storage, L, b->stream)
                    : kind == 1 ? launch_fused2_step(b->storage, L, b->stream)
                                : launch_fused4_step(b->storage, L, b->stream);
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
    const int per = kind == 1 ? 2 : 1;   // steps per launch
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
    long long done_clock = -1;
    while (b->marks.size() > 1 && cudaEventQuery(b->marks.front().second) == cudaSuccess) {
        done_clock = b->marks.front().first;
        b->free_marks.push_back(b->marks.front().second);
        b->marks.pop_front();
    }
    if (done_clock >= 0 && !b->retired_graphs.empty()) batch_free_finished_graphs(b, done_clock);
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
    for (int q = 0; q < 2; ++q) {
        cudaFreeHost(b->h_stage[q]);
        if (b->h_stage_ev[q]) cudaEventDestroy(b->h_stage_ev[q]);
    }
    cudaEventDestroy(b->done_ev);
    for (auto &mk : b->marks) cudaEventDestroy(mk.second);
    for (cudaEvent_t e : b->free_marks) cudaEventDestroy(e);
    delete b;
}

}  // extern "C"
