// fdtd_energy_static: the discrete Yee energy of caller-owned device fields,
// computed without allocating any device memory.
//
// Who needs it: callers that must not (or cannot) call cudaMalloc on the path
// where they want the energy -- a host loop that captures its work into a CUDA
// graph, a process that pre-reserved nearly all of HBM for its own arena and
// must not fail or fragment on a late allocation, or a latency-critical loop in
// which cudaMalloc's implicit device synchronisation is not acceptable.  They
// hand in their own device buffers for the inputs and the result; the partial
// sums live in a fixed array below.
//
// Scratch: g_energy_partial, one double per z-plane of the canonical grid
// (nz + 1 <= kStaticPlanes), a file-scope __device__ array that every GPU which
// loads this library holds until the process exits (64 KiB).  Each call writes
// all the entries it later reads (one per plane), so nothing has to be cleared
// between calls.  All calls share the array: calls whose kernels overlap on the
// GPU (different streams, or different host threads on the same device) race
// on it and must be serialised by the caller.
//
// The host side resolves the array's device address with cudaGetSymbolAddress
// once per device, with that device current, on the first call made on that
// device; that first call should therefore come before any stream capture.
// The address is remembered together with the CUDA context it belongs to: when
// the current context of the device is a different one (the primary context
// was reset with cudaDeviceReset and made again, which reloads the library's
// device code), the address is looked up again before the kernel is launched.
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "../../include/fdtd.h"
#include "launch.h"

namespace fdtd {

void set_last_error(const char *msg);   // ctx.cu: message returned by fdtd_last_error(NULL)

namespace {

constexpr int kStaticPlanes = 8192;     // nz + 1 <= 8192
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_partial[kStaticPlanes];

struct CanonArgs {
    const float *f[6];
    const float *coef[6];   // ce x,y,z then ch x,y,z; NULL = vacuum value
    float vac;
    int nx, ny, nz;
};

// One block per canonical z-plane k (0..nz): sum of E^2/ce + H (H - ch curl E)/ch over the
// positions of that plane inside each component's Yee extent, written to partial[k].
__global__ void __launch_bounds__(kThreads) energy_plane_kernel(const CanonArgs a, double *partial) {
    __shared__ double sh[kThreads / 32];
    const int k = blockIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long NX1 = nx + 1, NY1 = ny + 1;
    const long long zs = NX1 * NY1;
    auto F = [&](int c, long long q) -> double { return (double)a.f[c][q]; };
    auto C = [&](int c, long long q) -> double { return a.coef[c] ? (double)a.coef[c][q] : (double)a.vac; };
    double s = 0.0;
    for (long long p = threadIdx.x; p < zs; p += kThreads) {
        const int i = (int)(p % NX1), j = (int)(p / NX1);
        const long long q = (long long)k * zs + p;
        if (i < nx) s += F(0, q) * F(0, q) / C(0, q);
        if (j < ny) s += F(1, q) * F(1, q) / C(1, q);
        if (k < nz) s += F(2, q) * F(2, q) / C(2, q);
        if (j < ny && k < nz) {
            const double c = (F(2, q + NX1) - F(2, q)) - (F(1, q + zs) - F(1, q));
            const double h = F(3, q), ch = C(3, q);
            s += h * (h - ch * c) / ch;
        }
        if (i < nx && k < nz) {
            const double c = (F(0, q + zs) - F(0, q)) - (F(2, q + 1) - F(2, q));
            const double h = F(4, q), ch = C(4, q);
            s += h * (h - ch * c) / ch;
        }
        if (i < nx && j < ny) {
            const double c = (F(1, q + 1) - F(1, q)) - (F(0, q + NX1) - F(0, q));
            const double h = F(5, q), ch = C(5, q);
            s += h * (h - ch * c) / ch;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
        partial[k] = t;
    }
}

// Sum partial[0..n) in a fixed order and scale: W = 1/2 (dt/dx) sum.
__global__ void __launch_bounds__(kThreads) energy_final_kernel(const double *partial, int n, double scale, double *W) {
    __shared__ double sh[kThreads / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += kThreads) s += partial[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
        *W = scale * t;
    }
}

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};   // the context each cached address belongs to

// cuCtxGetCurrent from the driver (through the runtime's entry-point query, so the library links
// against no driver library); NULL when the driver does not offer it.
PFN_cuCtxGetCurrent_v4000 ctx_get_current() {
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    });
    return fn;
}

// Device address of g_energy_partial on the current device: resolved on the first call made on a
// device, and again whenever the device's current context is not the one it was resolved in.
cudaError_t scratch_address(double **out, int *dev_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    CUcontext cur = nullptr;
    auto get = ctx_get_current();
    if (!get || get(&cur) != CUDA_SUCCESS) return cudaErrorUnknown;
    std::lock_guard<std::mutex> g(g_mu);
    if (!cur || !g_scratch_addr[dev] || g_scratch_ctx[dev] != cur) {
        // no context current yet on this thread (cudaGetSymbolAddress makes the device's primary
        // context current), or another context than the cached address belongs to
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_energy_partial);
        if (e != cudaSuccess) return e;
        if (get(&cur) != CUDA_SUCCESS || !cur) return cudaErrorUnknown;
        g_scratch_addr[dev] = static_cast<double *>(p);
        g_scratch_ctx[dev] = cur;
    }
    *out = g_scratch_addr[dev];
    *dev_out = dev;
    return cudaSuccess;
}

int fail_static(int code, const std::string &msg) {
    set_last_error(msg.c_str());
    return code;
}

}  // namespace
}  // namespace fdtd

extern "C" int fdtd_energy_static(int nx, int ny, int nz, double dt, double dx, const float *const f[6],
                                  const float *const ce[3], const float *const ch[3], double *W,
                                  void *cuda_stream) {
    using namespace fdtd;
    if (!f || !W) return fail_static(FDTD_ERR_ARG, "fdtd_energy_static: NULL fields or result pointer");
    for (int c = 0; c < 6; ++c)
        if (!f[c]) return fail_static(FDTD_ERR_ARG, "fdtd_energy_static: a field pointer is NULL");
    if (nx < 1 || ny < 1 || nz < 1)
        return fail_static(FDTD_ERR_ARG, "fdtd_energy_static: cell counts must be >= 1");
    if ((long long)nz + 1 > kStaticPlanes)
        return fail_static(FDTD_ERR_ARG, "fdtd_energy_static: nz = " + std::to_string(nz) +
                                             " exceeds the static scratch limit of " +
                                             std::to_string(kStaticPlanes - 1) + " planes");
    if (((long long)nx + 1) * ((long long)ny + 1) > (1ll << 31))
        return fail_static(FDTD_ERR_ARG, "fdtd_energy_static: a z-plane has more than 2^31 points");
    if (!(dt > 0) || !(dx > 0)) return fail_static(FDTD_ERR_ARG, "fdtd_energy_static: dt and dx must be positive");
    const bool have_ce = ce && ce[0] && ce[1] && ce[2];
    const bool have_ch = ch && ch[0] && ch[1] && ch[2];
    if ((ce && !have_ce && (ce[0] || ce[1] || ce[2])) || (ch && !have_ch && (ch[0] || ch[1] || ch[2])))
        return fail_static(FDTD_ERR_ARG, "fdtd_energy_static: coefficient arrays must be all three or none");
    double *scratch = nullptr;
    int dev = 0;
    cudaError_t e = scratch_address(&scratch, &dev);
    if (e != cudaSuccess)
        return fail_static(FDTD_ERR_CUDA, std::string("fdtd_energy_static: cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e));
    CanonArgs a{};
    for (int c = 0; c < 6; ++c) a.f[c] = f[c];
    for (int c = 0; c < 3; ++c) {
        a.coef[c] = have_ce ? ce[c] : nullptr;
        a.coef[3 + c] = have_ch ? ch[c] : nullptr;
    }
    a.vac = (float)(dt / dx);
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    energy_plane_kernel<<<nz + 1, kThreads, 0, s>>>(a, scratch);
    energy_final_kernel<<<1, kThreads, 0, s>>>(scratch, nz + 1, 0.5 * dt / dx, W);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail_static(FDTD_ERR_CUDA, std::string("fdtd_energy_static: launch: ") + cudaGetErrorString(e));
    return FDTD_OK;
}
