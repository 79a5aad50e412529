// Point currents and field probes: one small launch after each step of a context that has them.
//
// Eq. 1 of the paper (Sec. 2) carries a current density J that the benchmark sets to zero; with J the
// E update of the step from E^n to E^{n+1} also subtracts ce * dx * J^{n+1/2} at the current's position.
// The step kernels compute E^{n+1} without it; this kernel then subtracts the source term (one rounding
// more than a fused form, well inside the FP32 tolerance) and records the probed components, in physical
// units, for the step whose index it reads from a device clock (so graph replays need no host update).
#include "fdtd_internal.cuh"
#include "launch.h"

namespace fdtd {

namespace {

template <typename T>
__global__ void extras_kernel(const CavityDesc d, int copy, const ExtrasParams X) {
    const long long n = *X.clock;   // index of the step just taken (counted from fdtd_set_fields)
    if (threadIdx.x == 0)
        for (int s = 0; s < X.nsrc; ++s) {   // serial: several currents may share a position
            const float J = n < X.wave_len ? X.wave[(size_t)s * X.wave_len + n] : 0.f;
            if (J == 0.f) continue;
            const int c = X.src_comp[s];
            const long long off = X.src_off[s];
            const float e = ld_field<T>(d, copy, c, off);
            st_field<T>(d, copy, c, off, e - (ld_coef(d, c, off) * X.dx) * J);
        }
    __syncthreads();
    const long long slot = n - X.probe_start;
    if (slot >= 0 && slot < X.capacity)
        for (int p = threadIdx.x; p < X.nprobe; p += blockDim.x)
            X.probe_buf[(size_t)p * X.capacity + slot] = ld_field<T>(d, copy, X.probe_comp[p], X.probe_off[p]);
    __syncthreads();
    if (threadIdx.x == 0) *X.clock = n + 1;
}

}  // namespace

cudaError_t launch_extras(int storage, const CavityDesc &d, int copy, const ExtrasParams &X, cudaStream_t s) {
    if (storage == 0)
        extras_kernel<float><<<1, 128, 0, s>>>(d, copy, X);
    else if (storage == 1)
        extras_kernel<__half><<<1, 128, 0, s>>>(d, copy, X);
    else
        extras_kernel<__nv_bfloat16><<<1, 128, 0, s>>>(d, copy, X);
    return cudaGetLastError();
}

}  // namespace fdtd
