// Point currents (the J of Eq. 1) and field probes of a single cavity: host-side validation, device
// arrays, and the small launch that follows every step while either is set.
#include "api_internal.h"

namespace fdtd {

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

}  // namespace fdtd

using namespace fdtd;

extern "C" {

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

}  // extern "C"
