// Launch planning of the fused kernels: launch shape from the tuning (tile height, ring depth,
// occupancy), the z-chunk plan with the shortest simulated makespan, the chunk-major tile list and
// its greedy assignment to the persistent CTAs, and the host-only diagnostic of that split.
#include "api_internal.h"

namespace fdtd {

// Launch shape of kernel kind 0 (one step) or 1 (two steps) from the tuning (invalid fields -> defaults).
Shape resolve_shape(int storage, const fdtd_tuning &t, int kind) {
    static std::mutex mu;
    static std::map<int, int> occ_cache;   // (kind, storage, tile_y, stages) -> max CTAs per SM
    Shape s;
    s.kind = kind;
    s.rows_per_warp = kind == 1 ? two_step_rows(t) : 1;
    const bool rows2 = s.rows_per_warp == 2;
    if (kind == 2)
        s.tile_y = (t.tile_y == 4 || t.tile_y == 8 || t.tile_y == 12 || t.tile_y == 16) ? t.tile_y : 12;
    else if (kind == 3)
        s.tile_y = (t.tile_y == 8 || t.tile_y == 10 || t.tile_y == 12) ? t.tile_y : 10;
    else if (kind == 0)
        s.tile_y = (t.tile_y == 4 || t.tile_y == 8 || t.tile_y == 16) ? t.tile_y : 8;
    else if (rows2)
        s.tile_y = (t.tile_y == 12 || t.tile_y == 16) ? t.tile_y : 16;
    else
        s.tile_y = (t.tile_y == 8 || t.tile_y == 12 || t.tile_y == 16) ? t.tile_y : 16;
    const int min_st = kind == 2 ? 4 : 3;
    // default ring depths: measured best at 512^3; the fourth-order kernel (three units resident) takes
    // the deepest ring that fits, which measured best for each of its tile heights
    s.stages = (t.stages >= min_st && t.stages <= 8) ? t.stages : (kind == 0 ? 4 : kind == 1 ? 6 : 8);   // kind 3: deepest
    auto smem = [&](int st) {
        return kind == 0   ? fused_smem_bytes(storage, s.tile_y, st)
               : kind == 1 ? (rows2 ? fused2r_smem_bytes(storage, s.tile_y, st) : fused2_smem_bytes(storage, s.tile_y, st))
               : kind == 3 ? fused3_smem_bytes(storage, s.tile_y, st)
                           : fused4_smem_bytes(storage, s.tile_y, st);
    };
    while (s.stages > min_st && smem(s.stages) > 227 * 1024) --s.stages;
    const int key = (((kind * 4 + storage) * 64 + s.tile_y) * 16 + s.stages) * 4 + s.rows_per_warp;
    int occ = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = occ_cache.find(key);
        if (it != occ_cache.end()) {
            occ = it->second;
        } else {
            cudaError_t e = kind == 0   ? fused_occupancy(storage, s.tile_y, s.stages, &occ)
                            : kind == 1 ? (rows2 ? fused2r_occupancy(storage, s.tile_y, s.stages, &occ)
                                                 : fused2_occupancy(storage, s.tile_y, s.stages, &occ))
                            : kind == 3 ? fused3_occupancy(storage, s.tile_y, s.stages, &occ)
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

TileRec base_rec(const fdtd_ctx *c, int parity_off, int set) {
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
    // the two-step map set reads the PEC-coded ids (encode_maps) and takes their table
    const bool pec = set == 1 && c->id_pec;
    r.table = reinterpret_cast<const float4 *>(pec ? c->table_pec : c->table_fused);
    r.ntab = pec ? c->ntab_pec : c->ntab;
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
    const int tw = kind == 1 ? fused2_tile_w(c->storage) : kind == 3 ? fused3_tile_w() : kTileX;
    int z0 = 0;
    for (int len : plan) {
        for (int y0 = 0; y0 < c->ny; y0 += tile_y)
            for (int x0 = 0; x0 < c->nx; x0 += tw) {
                TileRec t = b;
                t.x0 = x0;
                t.y0 = y0;
                t.kz0 = z0;
                t.kz1 = z0 + len;
                // two- and three-step kernels: 16-byte aligned origin of the id box (lane cells from x0 - 2,
                // resp. x0 - 4)
                t.id_x0 = (x0 - (kind == 3 ? 4 : 2)) & ~15;
                v.push_back(t);
            }
        z0 += len;
    }
}

void append_tiles(std::vector<TileRec> &v, const fdtd_ctx *c, int parity_off, int tile_y, int zlen, int kind) {
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
    const int tw = kind == 1 ? fused2_tile_w(c->storage) : kind == 3 ? fused3_tile_w() : kTileX;
    const long long cols = (long long)((c->nx + tw - 1) / tw) * ((c->ny + s.tile_y - 1) / s.tile_y);
    const int prologue = kind == 0 ? 1 : kind == 1 ? 3 : kind == 3 ? 5 : 4;
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


}  // namespace fdtd

using namespace fdtd;

extern "C" {

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

}  // extern "C"
