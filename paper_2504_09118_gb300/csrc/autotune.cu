// Autotuning of the step kernels: candidates timed on the caller's own state (copied aside and
// restored), a per-shape cache for single cavities, and the size-bucket model of online re-tuning
// for batches whose members change.
#include "api_internal.h"

namespace fdtd {

std::vector<fdtd_tuning> tune_candidates(bool batch, int order) {
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
    // single cavities: three steps per launch, deepest ring that fits
    if (!batch)
        for (int ty : {8, 10, 12}) v.push_back(fdtd_tuning{FDTD_KERNEL_TEMPORAL3, ty, 0, 0, 0, 1});
    // two rows per consumer warp, with the deepest ring that fits beside its smaller exchange planes
    for (int ty : {12, 16}) v.push_back(fdtd_tuning{FDTD_KERNEL_TEMPORAL2, ty, 0, 0, 0, 1});
    return v;
}

int trial_length(int trial_steps) {   // whole 16-step graphs
    const int n = trial_steps <= 0 ? 16 : trial_steps;
    return (n + 15) / 16 * 16;
}

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int, int>, std::pair<fdtd_tuning, double>> g_tune_cache;
}  // namespace

}  // namespace fdtd

using namespace fdtd;

extern "C" {

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
        for (const fdtd_tuning &t : tune_candidates(true, b->order)) {
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
    const auto key = std::make_pair(b->storage * 8 + b->order, floor_log2(cells));
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

}  // extern "C"
