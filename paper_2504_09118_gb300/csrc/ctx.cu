// C ABI of libfdtd, single cavities: context lifecycle, coefficient compression, layout conversion at
// load and read-back, step dispatch (fused TMA kernels with CUDA-graph replay, or the unfused
// baseline) and the FP64 reductions.
#include "api_internal.h"

namespace fdtd {

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
    d.kr_lo = 0;
    d.kr_hi = c->nz;
    d.face_top = 1;
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
    // field box width: one granule of halo on each side of the 64 lane cells, except for the two- and
    // three-step kernels, whose lane cells start left of the tile and whose box origin is rounded down to
    // the granule: 64 + one granule
    const int bx = (set == 1 || set == 3) ? kTileX + hx : kTileX + 2 * hx;
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
        // the two-step kernels read the PEC-coded ids when the context has them (their records then
        // carry table_pec)
        uint8_t *ids = set == 1 && c->id_pec ? c->id_pec : c->id;
        CUresult r = enc(&maps[12], CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, ids, gdim, gstr, box, estr,
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
           (c->tuning.kernel == FDTD_KERNEL_TEMPORAL || c->tuning.kernel == FDTD_KERNEL_TEMPORAL2 ||
            c->tuning.kernel == FDTD_KERNEL_TEMPORAL3 || c->tuning.kernel == FDTD_KERNEL_AUTO);
}

// Steps per launch of the context's multi-step kernel (use_temporal): 3 for TEMPORAL3, else 2.
static int temporal_steps(const fdtd_ctx *c) { return c->tuning.kernel == FDTD_KERNEL_TEMPORAL3 ? 3 : 2; }

// Tile kind of a context's one-step launches: 0 (Eq. 2) or 2 (fourth order).
int one_step_kind(const fdtd_ctx *c) { return c->order == 4 ? 2 : 0; }

// One launch of a single context (no graph): kinds 0 and 2 advance one step, kind 1 two steps.
int launch_one(fdtd_ctx *c, int parity, int inject_us, int kind) {
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
    L.rows_per_warp = s.rows_per_warp;
    L.coef_class = coef_class_of(c->coef_mode, c->ch_uniform, kind == 1 && c->id_pec);
    if (kind == 0)
        CK(c, launch_fused_step(c->storage, L, c->stream));
    else if (kind == 1)
        CK(c, launch_fused2_step(c->storage, L, c->stream));
    else if (kind == 3)
        CK(c, launch_fused3_step(c->storage, L, c->stream));
    else
        CK(c, launch_fused4_step(c->storage, L, c->stream));
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


namespace {
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

// PEC as materials.  tab: ntab entries of 8 floats (ce xyz, pad, ch xyz, pad), as folded for the fused
// kernels.  Entry 1 + m + ntab f is material m on the faces f (bit 0: i = 0, bit 1: j = 0, bit 2: k = 0)
// with the E coefficients of the components tangential to those faces set to zero (Ex lies in the
// j = 0 and k = 0 faces, Ey in i = 0 and k = 0, Ez in i = 0 and j = 0), so that an update with that
// entry keeps them at their initial zero.  Entry 0 is what a TMA box reads outside the cavity: ce = 0
// (E there stays the 0 it was read as) and material 0's ch.  Face-major order keeps the interior
// entries (f = 0) of all materials adjacent, 32 bytes apart, as in the plain table: lanes of a warp
// that read different materials then hit different shared-memory banks.
// PEC-coded id of a cell of material id on the faces it lies on (entry 1 + id + ntab f of pec_table).
int pec_code(int id, int ntab, int i, int j, int k) {
    const int faces = (i == 0 ? 1 : 0) + (j == 0 ? 2 : 0) + (k == 0 ? 4 : 0);
    return 1 + id + ntab * faces;
}

std::vector<float> pec_table(const std::vector<float> &tab, int ntab) {
    std::vector<float> t(8 * kMaxTable, 0.f);
    for (int q = 0; q < 3; ++q) t[4 + q] = tab[4 + q];
    for (int m = 0; m < ntab; ++m)
        for (int f = 0; f < 8; ++f) {
            float *e = &t[8 * (1 + m + ntab * f)];
            const bool i0 = f & 1, j0 = f & 2, k0 = f & 4;
            e[0] = (j0 || k0) ? 0.f : tab[8 * m + 0];
            e[1] = (i0 || k0) ? 0.f : tab[8 * m + 1];
            e[2] = (i0 || j0) ? 0.f : tab[8 * m + 2];
            for (int q = 0; q < 3; ++q) e[4 + q] = tab[8 * m + 4 + q];
        }
    return t;
}

}  // namespace

// Message returned by fdtd_last_error(NULL) on this thread (used by context-free entry points).
void set_last_error(const char *msg) { g_create_error = msg; }

}  // namespace fdtd

using namespace fdtd;

extern "C" {

const char *fdtd_version(void) { return "fdtd-gb300 0.1 (sm_103a)"; }

int fdtd_debug_pec_code(int ntab, int id, int i, int j, int k, int *code) {
    if (!code || ntab < 1 || ntab > kMaxPecMaterials || id < 0 || id >= ntab || i < 0 || j < 0 || k < 0)
        return FDTD_ERR_ARG;
    *code = pec_code(id, ntab, i, j, k);
    return FDTD_OK;
}

int fdtd_debug_pec_table(const float *tab, int ntab, float *out) {
    if (!tab || !out || ntab < 1 || ntab > kMaxPecMaterials) return FDTD_ERR_ARG;
    const std::vector<float> t = pec_table(std::vector<float>(tab, tab + 8 * ntab), ntab);
    std::copy(t.begin(), t.begin() + 8 * (1 + 8 * ntab), out);
    return FDTD_OK;
}

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
            if (c->ntab <= kMaxPecMaterials) {
                // PEC as materials for the two-step kernel: the face a cell lies on selects its table entry
                std::vector<uint8_t> pec(ids.size());
                for (int k = 0; k < nz; ++k)
                    for (int j = 0; j < ny; ++j)
                        for (int i = 0; i < nx; ++i) {
                            const size_t q = ((size_t)k * ny + j) * nx + i;
                            pec[q] = (uint8_t)pec_code(ids[q], c->ntab, i, j, k);
                        }
                if ((e = dmalloc(c, (void **)&c->id_pec, c->arr_elems)) != cudaSuccess) return cfail("id alloc", e);
                if ((e = cudaMemset(c->id_pec, 0, c->arr_elems)) != cudaSuccess) return cfail("memset", e);
                if ((e = cudaMemcpy2D(c->id_pec, c->pitch, pec.data(), nx, nx, (size_t)ny * nz,
                                      cudaMemcpyHostToDevice)) != cudaSuccess)
                    return cfail("id copy", e);
                const std::vector<float> tp = pec_table(tab, c->ntab);
                if ((e = dmalloc(c, (void **)&c->table_pec, tp.size() * 4)) != cudaSuccess)
                    return cfail("table alloc", e);
                if ((e = cudaMemcpy(c->table_pec, tp.data(), tp.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
                    return cfail("table copy", e);
                c->ntab_pec = 1 + 8 * c->ntab;
            }
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
    for (void *p : {(void *)c->id, (void *)c->id_pec, (void *)c->table_pec, (void *)c->table, (void *)c->inv_table,
                    (void *)c->table_fused,
                    (void *)c->d_status, (void *)c->d_partial, (void *)c->d_out, (void *)c->d_stage,
                    (void *)c->d_max, (void *)c->d_maps, (void *)c->d_desc, (void *)c->tl[0].d,
                    (void *)c->tl[1].d, (void *)c->tl[2].d, (void *)c->tl[3].d, (void *)c->d_src_comp, (void *)c->d_src_off, (void *)c->d_wave,
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
    if (c->slab.ev) cudaEventDestroy(c->slab.ev);
    if (c->prefetch_free) cudaEventDestroy(c->prefetch_free);
    delete c;
}

long long fdtd_steps_done(const fdtd_ctx *c) { return c ? c->steps : -1; }
long long fdtd_device_bytes(const fdtd_ctx *c) { return c ? c->bytes : -1; }

int fdtd_set_tuning(fdtd_ctx *c, const fdtd_tuning *t) {
    if (!c) return FDTD_ERR_ARG;
    fdtd_tuning n{};
    if (t) n = *t;
    if (n.kernel < 0 || n.kernel > FDTD_KERNEL_TEMPORAL3) return fail(c, FDTD_ERR_ARG, "bad kernel %d", n.kernel);
    const bool two_step = n.kernel == FDTD_KERNEL_TEMPORAL || n.kernel == FDTD_KERNEL_TEMPORAL2 ||
                          n.kernel == FDTD_KERNEL_TEMPORAL3;
    if (two_step && c->order != 2)
        return fail(c, FDTD_ERR_ARG, "the two-step kernels run the second-order scheme only");
    // one-step kernels: 4, 8 or 16 rows (the fourth-order kernel also 12); two-step kernel: 8, 12 or 16;
    // two-step kernel with two rows per warp: 12 or 16
    const bool ty_one = n.tile_y == 4 || n.tile_y == 8 || n.tile_y == 16 || (c->order == 4 && n.tile_y == 12),
               ty_two = n.tile_y == 8 || n.tile_y == 12 || n.tile_y == 16, ty_two2 = n.tile_y == 12 || n.tile_y == 16;
    if (n.tile_y && !(n.kernel == FDTD_KERNEL_TEMPORAL    ? ty_two
                      : n.kernel == FDTD_KERNEL_TEMPORAL2 ? ty_two2
                      : n.kernel == FDTD_KERNEL_TEMPORAL3 ? (n.tile_y == 8 || n.tile_y == 10 || n.tile_y == 12)
                      : n.kernel == FDTD_KERNEL_AUTO      ? (ty_one || ty_two)
                                                          : ty_one))
        return fail(c, FDTD_ERR_ARG, "tile_y must be 4, 8 or 16 (fourth order: also 12; two-step kernel: 8, 12 or 16; "
                                     "two-step kernel with two rows per warp: 12 or 16; three-step kernel: 8, 10 or 12)");
    if (n.stages && (n.stages < 3 || n.stages > 8)) return fail(c, FDTD_ERR_ARG, "stages must be in [3, 8]");
    if (n.stages == 3 && c->order == 4) return fail(c, FDTD_ERR_ARG, "the fourth-order kernel needs stages >= 4");
    if (n.zchunk < 0 || n.ctas_per_sm < 0) return fail(c, FDTD_ERR_ARG, "negative tuning value");
    c->tuning = n;
    c->tl[0].key = c->tl[1].key = c->tl[2].key = c->tl[3].key = 0;   // force tile rebuilds
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
    if (order == 4 && (c->tuning.kernel == FDTD_KERNEL_TEMPORAL || c->tuning.kernel == FDTD_KERNEL_TEMPORAL2 ||
                       c->tuning.kernel == FDTD_KERNEL_TEMPORAL3))
        return fail(c, FDTD_ERR_ARG, "the multi-step kernels run the second-order scheme only; retune first");
    if (order == 4 && c->tuning.stages == 3)
        return fail(c, FDTD_ERR_ARG, "the fourth-order kernel needs stages >= 4; retune first");
    cudaStreamSynchronize(c->stream);   // no graph of this context may still be running
    drop_graphs(c->graphs);
    c->order = order;
    slab_after_load(c);   // the ghost depth a step needs changed with the reach of the differences
    return FDTD_OK;
}

int fdtd_get_order(const fdtd_ctx *c) { return c ? c->order : -1; }

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
            float sc = mx > 0.f ? std::ldexp(1.0f, 8 - (int)std::ceil(std::log2((double)mx))) : 1.0f;
            if (c->fixed_scale[g] > 0.f) {   // fdtd_set_storage_scales
                sc = c->fixed_scale[g];
                if (c->storage == FDTD_F16 && (double)mx * sc > 60000.0)
                    return fail(c, FDTD_ERR_ARG, "fixed storage scale %g overflows FP16 for |%s| up to %g", sc,
                                g ? "H" : "E", (double)mx);
            }
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
            if (c->table_pec) {
                const std::vector<float> tp = pec_table(tf, c->ntab);
                CK(c, cudaMemcpyAsync(c->table_pec, tp.data(), tp.size() * 4, cudaMemcpyHostToDevice, c->stream));
                CK(c, cudaStreamSynchronize(c->stream));
            }
        }
        c->tl[0].key = c->tl[1].key = c->tl[2].key = c->tl[3].key = 0;   // tile records embed the folded coefficients
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
    slab_after_load(c);
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
    if (int rc = slab_check_steps(c, nsteps)) return rc;
    const bool fused = use_fused(c);
    const bool extras = extras_on(c);
    // currents enter between the E update of one step and the H update of the next: one step per launch
    const bool temporal = use_temporal(c) && !extras;
    const int k1 = one_step_kind(c);
    if (fused)
        if (int rc = build_tiles(c, k1)) return rc;
    // kind 1 (two steps per launch) or 3 (three steps per launch)
    const int tkind = temporal_steps(c) == 3 ? 3 : 1, tper = temporal_steps(c);
    if (temporal)
        if (int rc = build_tiles(c, tkind)) return rc;
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
    // kind 1 advances two steps per launch, kind 3 three; every fused kind reads copy cur and writes copy
    // 1 - cur.  A remainder takes launches of the one-step kernel at the end.
    const int kind = temporal ? tkind : k1;
    const int per = temporal ? tper : 1;
    const int K = per == 3 ? 18 : 16;   // steps per graph: an even number of launches
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
        for (; left >= tper; left -= tper) {
            if (int rc = step_launch(c->cur, 0, tkind)) return rc;
            c->cur ^= 1;
            c->steps += tper;
        }
    for (; left > 0; --left) {
        if (int rc = step_launch(c->cur, 0, k1)) return rc;
        if (fused) c->cur ^= 1;
        ++c->steps;
    }
    slab_took_steps(c, nsteps);
    return FDTD_OK;
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

}  // extern "C"
