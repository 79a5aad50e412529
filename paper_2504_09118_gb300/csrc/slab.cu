// z-slab decomposition of one cavity (domain decomposition, named in Sec. 6 of the paper): a slab
// context owns the cells of global planes [k0, k1) and keeps `ghost` extra cells on each side that has
// a neighbouring slab.  Its kernels are the ordinary ones, so on a ghost side they treat the local
// boundary as a PEC wall: wrong there, and the error moves inwards by the reach of the scheme per step
// (one plane for Eq. 2, three for the fourth-order differences).  After an exchange that copies `ghost`
// cells of all six fields from the neighbours, the owned cells therefore stay exact for
// floor(ghost / reach) steps; fdtd_step refuses more.  Every owned value is computed by the same
// operations from the same inputs as in one undivided cavity, so FP32 results agree bit for bit (and
// 16-bit ones too when every slab uses the same storage scales, fdtd_set_storage_scales).
#include "api_internal.h"

namespace fdtd {

int slab_reach(const fdtd_ctx *c) { return c->order == 4 ? 3 : 1; }

static int slab_budget(const fdtd_ctx *c) { return c->slab.ghost / slab_reach(c); }

void slab_after_load(fdtd_ctx *c) {
    if (!c->slab.on) return;
    // a load (or a change of the scheme) leaves the ghost cells untrusted until the next import
    c->slab.left[0] = c->slab.g_lo > 0 ? 0 : INT_MAX;
    c->slab.left[1] = c->slab.g_hi > 0 ? 0 : INT_MAX;
}

int slab_check_steps(fdtd_ctx *c, int nsteps) {
    if (!c->slab.on) return FDTD_OK;
    const int left = std::min(c->slab.left[0], c->slab.left[1]);
    if (nsteps > left)
        return fail(c, FDTD_ERR_STATE,
                    "slab: %d steps asked, the ghost cells cover %d more (ghost %d, reach %d per step): "
                    "exchange with the neighbouring slabs first",
                    nsteps, left, c->slab.ghost, slab_reach(c));
    return FDTD_OK;
}

void slab_took_steps(fdtd_ctx *c, int nsteps) {
    if (!c->slab.on) return;
    for (int s = 0; s < 2; ++s)
        if (c->slab.left[s] != INT_MAX) c->slab.left[s] -= nsteps;
}

namespace {

// First local plane of the cells a side exports (its owned boundary cells) or imports (its ghosts).
int export_plane(const fdtd_ctx *c, int side) {
    return side == 0 ? c->slab.g_lo : c->nz - c->slab.g_hi - c->slab.ghost;
}
int import_plane(const fdtd_ctx *c, int side) { return side == 0 ? 0 : c->nz - c->slab.g_hi; }

size_t halo_plane_bytes(const fdtd_ctx *c) { return (size_t)c->pitch * c->ny * esize(c->storage); }

int check_side(fdtd_ctx *c, int side) {
    if (!c->slab.on) return fail(c, FDTD_ERR_STATE, "not a slab context (fdtd_create_slab)");
    if (side != 0 && side != 1) return fail(c, FDTD_ERR_ARG, "side must be 0 (below) or 1 (above)");
    if ((side == 0 ? c->slab.g_lo : c->slab.g_hi) == 0)
        return fail(c, FDTD_ERR_ARG, "side %d of this slab is a PEC wall of the cavity: nothing to exchange", side);
    if (!c->has_fields) return fail(c, FDTD_ERR_STATE, "fdtd_set_fields has not been called");
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member");
    return FDTD_OK;
}

// The six fields of `ghost` planes starting at local plane k of copy `copy`, as one strided copy:
// field f's planes are contiguous (ghost * pitch * ny elements) and the fields lie arr_elems apart.
cudaError_t copy_planes(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, cudaMemcpyKind kind,
                        cudaStream_t s) {
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, 6, kind, s);
}

bool current(const fdtd_ctx *c) {
    const int full = slab_budget(c);
    return (c->slab.g_lo == 0 || c->slab.left[0] == full) && (c->slab.g_hi == 0 || c->slab.left[1] == full);
}

}  // namespace
}  // namespace fdtd

using namespace fdtd;

extern "C" {

int fdtd_create_slab(fdtd_ctx **out, int nx, int ny, int nz_global, int k0, int k1, int ghost, double dt, double dx,
                     const float *const ce[3], const float *const ch[3], int storage, void *cuda_stream) {
    if (!out) return fail(nullptr, FDTD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nz_global < 1 || k0 < 0 || k1 > nz_global || k0 >= k1)
        return fail(nullptr, FDTD_ERR_ARG, "slab planes [%d, %d) are not a non-empty part of [0, %d)", k0, k1,
                    nz_global);
    if (ghost < 1 || ghost > 64) return fail(nullptr, FDTD_ERR_ARG, "ghost must be in [1, 64], got %d", ghost);
    const int g_lo = k0 > 0 ? ghost : 0, g_hi = k1 < nz_global ? ghost : 0;
    if (k0 - g_lo < 0 || k1 + g_hi > nz_global)
        return fail(nullptr, FDTD_ERR_ARG, "the ghost cells of slab [%d, %d) reach outside the cavity", k0, k1);
    if ((g_lo || g_hi) && k1 - k0 < ghost)
        return fail(nullptr, FDTD_ERR_ARG, "a slab must own at least `ghost` (%d) planes, got %d", ghost, k1 - k0);
    const int nz_loc = k1 - k0 + g_lo + g_hi;
    fdtd_ctx *c = nullptr;
    if (int rc = fdtd_create(&c, nx, ny, nz_loc, dt, dx, ce, ch, storage, cuda_stream)) return rc;
    c->slab.on = 1;
    c->slab.nz_global = nz_global;
    c->slab.z_off = k0 - g_lo;
    c->slab.g_lo = g_lo;
    c->slab.g_hi = g_hi;
    c->slab.ghost = ghost;
    // the exchange's ordering event belongs to the slab's device, which is current here
    if (cudaEventCreateWithFlags(&c->slab.ev, cudaEventDisableTiming) != cudaSuccess) {
        fdtd_destroy(c);
        return fail(nullptr, FDTD_ERR_CUDA, "slab event create failed");
    }
    slab_after_load(c);
    *out = c;
    return FDTD_OK;
}

int fdtd_slab_info(const fdtd_ctx *c, int info[7]) {
    if (!c || !info) return FDTD_ERR_ARG;
    if (!c->slab.on) return FDTD_ERR_STATE;
    info[0] = c->slab.nz_global;
    info[1] = c->slab.z_off + c->slab.g_lo;            // k0
    info[2] = c->slab.z_off + c->nz - c->slab.g_hi;    // k1
    info[3] = c->slab.g_lo;
    info[4] = c->slab.g_hi;
    info[5] = c->slab.ghost;
    info[6] = std::min(c->slab.left[0], c->slab.left[1]);
    return FDTD_OK;
}

long long fdtd_slab_halo_bytes(const fdtd_ctx *c) {
    if (!c || !c->slab.on) return -1;
    return 6ll * c->slab.ghost * (long long)halo_plane_bytes(c);
}

int fdtd_slab_export(fdtd_ctx *c, int side, void *buf, int on_device) {
    NvtxRange nvtx_range("fdtd_slab_export");
    if (!c || !buf) return fail(c, FDTD_ERR_ARG, "NULL argument");
    if (int rc = check_side(c, side)) return rc;
    const size_t pb = halo_plane_bytes(c), width = pb * c->slab.ghost, es = esize(c->storage);
    const char *src = static_cast<const char *>(c->fields[c->cur][0]) + (size_t)export_plane(c, side) * pb;
    CK(c, copy_planes(buf, width, src, c->arr_elems * es, width,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream));
    return FDTD_OK;
}

int fdtd_slab_import(fdtd_ctx *c, int side, const void *buf, int on_device) {
    NvtxRange nvtx_range("fdtd_slab_import");
    if (!c || !buf) return fail(c, FDTD_ERR_ARG, "NULL argument");
    if (int rc = check_side(c, side)) return rc;
    const size_t pb = halo_plane_bytes(c), width = pb * c->slab.ghost, es = esize(c->storage);
    char *dst = static_cast<char *>(c->fields[c->cur][0]) + (size_t)import_plane(c, side) * pb;
    CK(c, copy_planes(dst, c->arr_elems * es, buf, width, width,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (!on_device) CK(c, cudaStreamSynchronize(c->stream));
    c->slab.left[side] = slab_budget(c);
    return FDTD_OK;
}

int fdtd_slab_exchange(fdtd_ctx *lo, fdtd_ctx *hi) {
    NvtxRange nvtx_range("fdtd_slab_exchange");
    if (!lo || !hi || lo == hi) return fail(lo, FDTD_ERR_ARG, "two distinct slab contexts are needed");
    if (int rc = check_side(lo, 1)) return rc;
    if (int rc = check_side(hi, 0)) return rc;
    if (lo->nx != hi->nx || lo->ny != hi->ny || lo->storage != hi->storage || lo->slab.ghost != hi->slab.ghost ||
        lo->slab.nz_global != hi->slab.nz_global)
        return fail(lo, FDTD_ERR_ARG, "slabs differ in nx, ny, storage, ghost depth or cavity");
    if (lo->slab.z_off + lo->nz - lo->slab.g_hi != hi->slab.z_off + hi->slab.g_lo)
        return fail(lo, FDTD_ERR_ARG, "the slabs are not neighbours (k1 of the lower one != k0 of the upper one)");
    if (lo->scale[0] != hi->scale[0] || lo->scale[3] != hi->scale[3])
        return fail(lo, FDTD_ERR_ARG, "16-bit slabs need equal storage scales (fdtd_set_storage_scales)");
    // both copies run on lo's stream after hi's earlier work; hi's later work waits for them
    CK(lo, cudaEventRecord(hi->slab.ev, hi->stream));
    CK(lo, cudaStreamWaitEvent(lo->stream, hi->slab.ev, 0));
    // the six arrays of a copy lie arr_elems apart, and arr_elems differs between slabs of different depth
    const size_t pb = halo_plane_bytes(lo), width = pb * lo->slab.ghost;
    const size_t sp_lo = lo->arr_elems * esize(lo->storage), sp_hi = hi->arr_elems * esize(hi->storage);
    const char *lo_own = static_cast<const char *>(lo->fields[lo->cur][0]) + (size_t)export_plane(lo, 1) * pb;
    char *lo_ghost = static_cast<char *>(lo->fields[lo->cur][0]) + (size_t)import_plane(lo, 1) * pb;
    const char *hi_own = static_cast<const char *>(hi->fields[hi->cur][0]) + (size_t)export_plane(hi, 0) * pb;
    char *hi_ghost = static_cast<char *>(hi->fields[hi->cur][0]) + (size_t)import_plane(hi, 0) * pb;
    CK(lo, cudaMemcpy2DAsync(hi_ghost, sp_hi, lo_own, sp_lo, width, 6, cudaMemcpyDefault, lo->stream));
    CK(lo, cudaMemcpy2DAsync(lo_ghost, sp_lo, hi_own, sp_hi, width, 6, cudaMemcpyDefault, lo->stream));
    CK(lo, cudaEventRecord(lo->slab.ev, lo->stream));
    CK(lo, cudaStreamWaitEvent(hi->stream, lo->slab.ev, 0));
    lo->slab.left[1] = slab_budget(lo);
    hi->slab.left[0] = slab_budget(hi);
    return FDTD_OK;
}

// Owned-cell sums of a slab (the caller adds them over slabs): energy W (with its 1/2 dt/dx factor)
// and the squared divergences.  The ghost cells must be current (no step since the last exchange).
static int slab_reduce(fdtd_ctx *c, int what, double out[3]) {
    if (!c) return FDTD_ERR_ARG;
    if (!c->slab.on) return fail(c, FDTD_ERR_STATE, "not a slab context (fdtd_create_slab)");
    if (!c->has_fields) return fail(c, FDTD_ERR_STATE, "fdtd_set_fields has not been called");
    if (c->batch) return fail(c, FDTD_ERR_STATE, "context is a batch member");
    if (!current(c)) return fail(c, FDTD_ERR_STATE, "slab: exchange the ghost cells before a reduction");
    CavityDesc d = make_desc(c, 0);
    d.kr_lo = c->slab.g_lo;
    d.kr_hi = c->nz - c->slab.g_hi;
    d.face_top = c->slab.g_hi == 0;
    CK(c, launch_reductions(c->storage, d, c->cur, what, c->d_partial, reduction_blocks(), c->d_out, c->stream,
                            c->order));
    CK(c, cudaMemcpyAsync(out, c->d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return check_status(c, c->d_status, c->stream);
}

int fdtd_slab_energy(fdtd_ctx *c, double *W) {
    if (!W) return fail(c, FDTD_ERR_ARG, "NULL argument");
    double o[3];
    if (int rc = slab_reduce(c, 0, o)) return rc;
    *W = 0.5 * (c->dt / c->dx) * o[0];
    return FDTD_OK;
}

int fdtd_slab_divergence_sq(fdtd_ctx *c, double *divE2, double *divH2) {
    if (!divE2 || !divH2) return fail(c, FDTD_ERR_ARG, "NULL argument");
    double o[3];
    if (int rc = slab_reduce(c, 1, o)) return rc;
    *divE2 = o[1];
    *divH2 = o[2];
    return FDTD_OK;
}

int fdtd_set_storage_scales(fdtd_ctx *c, double s_e, double s_h) {
    if (!c) return FDTD_ERR_ARG;
    for (double s : {s_e, s_h}) {
        int e = 0;
        if (s != 0.0 && !(s > 0.0 && std::frexp(s, &e) == 0.5 && e > -100 && e < 100))
            return fail(c, FDTD_ERR_ARG, "storage scales must be 0 (chosen from the data) or powers of two");
    }
    c->fixed_scale[0] = (float)s_e;
    c->fixed_scale[1] = (float)s_h;
    return FDTD_OK;
}

double fdtd_storage_scale_of(double maxabs) {
    if (!(maxabs > 0.0) || !std::isfinite(maxabs)) return 1.0;
    return std::ldexp(1.0, 8 - (int)std::ceil(std::log2(maxabs)));
}

}  // extern "C"
