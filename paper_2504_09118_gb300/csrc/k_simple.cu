// Layout conversion, the unfused one-thread-per-cell Yee step, and the FP64
// energy/divergence reductions.
//
// The unfused step is two launches per step (Listing 1: curl H components,
// then curl E components), each updating one copy of the fields in place; it
// is the debugging baseline of the fused kernel and the path for coefficient
// sets too varied for a one-byte material id (COEF_FULL).
#include "df.cuh"
#include "launch.h"

namespace fdtd {

namespace {

constexpr int BXs = 32, BYs = 8;

__device__ __forceinline__ bool tangential(int comp, int i, int j, int k) {
    return (comp == 0 && (j == 0 || k == 0)) || (comp == 1 && (i == 0 || k == 0)) ||
           (comp == 2 && (i == 0 || j == 0));
}

// Planes per thread of the layout kernels: their loads are issued together before the stores, so that a
// thread keeps several DRAM reads in flight (one element per thread left these kernels latency-bound).
constexpr int KZs = 4;

template <typename T>
__device__ __forceinline__ void pack_one(const CavityDesc &d, int copy, int comp, float v, int i, int j, int k,
                                         float *face) {
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    if (i < nx && j < ny && k < nz) {
        if (comp < 3 && tangential(comp, i, j, k)) v = 0.f;
        st_field<T>(d, copy, comp, (long long)k * d.plane + (long long)j * d.pitch + i, v);
        return;
    }
    // far-face normal H: store the value after the same storage rounding
    float q = v;
    if (Storage<T>::scaled) q = Storage<T>::load(Storage<T>::store(v * d.scale[comp])) * d.inv_scale[comp];
    if (comp == 3 && i == nx && j < ny && k < nz) face[(long long)k * ny + j] = q;
    if (comp == 4 && j == ny && i < nx && k < nz) face[(long long)k * nx + i] = q;
    if (comp == 5 && k == nz && i < nx && j < ny) face[(long long)j * nx + i] = q;
}

// Canonical component -> active layout (and far faces); each thread takes KZs planes of one (i, j).
template <typename T>
__global__ void pack_kernel(const CavityDesc d, int copy, int comp, const float *__restrict__ canon, float *face) {
    const int i = blockIdx.x * BXs + threadIdx.x, j = blockIdx.y * BYs + threadIdx.y, k0 = blockIdx.z * KZs;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    if (i > nx || j > ny) return;
    const long long zs = (long long)(ny + 1) * (nx + 1), base = (long long)j * (nx + 1) + i;
    float v[KZs];
#pragma unroll
    for (int q = 0; q < KZs; ++q) v[q] = k0 + q <= nz ? canon[(k0 + q) * zs + base] : 0.f;
#pragma unroll
    for (int q = 0; q < KZs; ++q)
        if (k0 + q <= nz) pack_one<T>(d, copy, comp, v[q], i, j, k0 + q, face);
}

template <typename T>
__device__ __forceinline__ float unpack_one(const CavityDesc &d, int copy, int comp, int i, int j, int k) {
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    if (i < nx && j < ny && k < nz) return ld_field<T>(d, copy, comp, (long long)k * d.plane + (long long)j * d.pitch + i);
    if (comp == 3 && i == nx && j < ny && k < nz) return d.face[0][(long long)k * ny + j];
    if (comp == 4 && j == ny && i < nx && k < nz) return d.face[1][(long long)k * nx + i];
    if (comp == 5 && k == nz && i < nx && j < ny) return d.face[2][(long long)j * nx + i];
    return 0.f;
}

// Active layout (and far faces) -> canonical component, zero outside the extent; KZs planes per thread.
template <typename T>
__global__ void unpack_kernel(const CavityDesc d, int copy, int comp, float *__restrict__ canon) {
    const int i = blockIdx.x * BXs + threadIdx.x, j = blockIdx.y * BYs + threadIdx.y, k0 = blockIdx.z * KZs;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    if (i > nx || j > ny) return;
    const long long zs = (long long)(ny + 1) * (nx + 1), base = (long long)j * (nx + 1) + i;
    float v[KZs];
#pragma unroll
    for (int q = 0; q < KZs; ++q) v[q] = k0 + q <= nz ? unpack_one<T>(d, copy, comp, i, j, k0 + q) : 0.f;
#pragma unroll
    for (int q = 0; q < KZs; ++q)
        if (k0 + q <= nz) canon[(k0 + q) * zs + base] = v[q];
}

__device__ __forceinline__ bool in_extent(int comp, int i, int j, int k, int nx, int ny, int nz) {
    switch (comp) {
        case 0: return i < nx;
        case 1: return j < ny;
        case 2: return k < nz;
        case 3: return j < ny && k < nz;
        case 4: return i < nx && k < nz;
        default: return i < nx && j < ny;
    }
}

__global__ void maxabs_kernel(const float *__restrict__ canon, int comp, int nx, int ny, int nz, unsigned *out) {
    const int i = blockIdx.x * BXs + threadIdx.x, j = blockIdx.y * BYs + threadIdx.y, k = blockIdx.z;
    float v = 0.f;
    if (i <= nx && j <= ny && in_extent(comp, i, j, k, nx, ny, nz))
        v = fabsf(canon[((long long)k * (ny + 1) + j) * (nx + 1) + i]);
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(out, __float_as_uint(v));
}

// H^{n+1/2} = H^{n-1/2} - ch curl E^n, one thread per cell (E beyond the active range is 0).
template <typename T>
__global__ void simple_h_kernel(const CavityDesc d, int copy) {
    const int i = blockIdx.x * BXs + threadIdx.x, j = blockIdx.y * BYs + threadIdx.y, k = blockIdx.z;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    if (i >= nx || j >= ny) return;
    const long long P = d.pitch, Z = d.plane;
    const long long o = (long long)k * Z + (long long)j * P + i;
    const float ex = ld_field<T>(d, copy, 0, o), ey = ld_field<T>(d, copy, 1, o), ez = ld_field<T>(d, copy, 2, o);
    const float ex_j1 = j + 1 < ny ? ld_field<T>(d, copy, 0, o + P) : 0.f;
    const float ex_k1 = k + 1 < nz ? ld_field<T>(d, copy, 0, o + Z) : 0.f;
    const float ey_i1 = i + 1 < nx ? ld_field<T>(d, copy, 1, o + 1) : 0.f;
    const float ey_k1 = k + 1 < nz ? ld_field<T>(d, copy, 1, o + Z) : 0.f;
    const float ez_i1 = i + 1 < nx ? ld_field<T>(d, copy, 2, o + 1) : 0.f;
    const float ez_j1 = j + 1 < ny ? ld_field<T>(d, copy, 2, o + P) : 0.f;
    const float hx = ld_field<T>(d, copy, 3, o) - ld_coef(d, 3, o) * ((ez_j1 - ez) - (ey_k1 - ey));
    const float hy = ld_field<T>(d, copy, 4, o) - ld_coef(d, 4, o) * ((ex_k1 - ex) - (ez_i1 - ez));
    const float hz = ld_field<T>(d, copy, 5, o) - ld_coef(d, 5, o) * ((ey_i1 - ey) - (ex_j1 - ex));
    st_field<T>(d, copy, 3, o, hx);
    st_field<T>(d, copy, 4, o, hy);
    st_field<T>(d, copy, 5, o, hz);
}

// E^{n+1} = E^n + ce curl H^{n+1/2} on entries not tangential to a face.
template <typename T>
__global__ void simple_e_kernel(const CavityDesc d, int copy) {
    const int i = blockIdx.x * BXs + threadIdx.x, j = blockIdx.y * BYs + threadIdx.y, k = blockIdx.z;
    const int nx = d.nx, ny = d.ny;
    if (i >= nx || j >= ny) return;
    const long long P = d.pitch, Z = d.plane;
    const long long o = (long long)k * Z + (long long)j * P + i;
    const float hx = ld_field<T>(d, copy, 3, o), hy = ld_field<T>(d, copy, 4, o), hz = ld_field<T>(d, copy, 5, o);
    if (j >= 1 && k >= 1) {
        const float c = (hz - ld_field<T>(d, copy, 5, o - P)) - (hy - ld_field<T>(d, copy, 4, o - Z));
        st_field<T>(d, copy, 0, o, ld_field<T>(d, copy, 0, o) + ld_coef(d, 0, o) * c);
    }
    if (i >= 1 && k >= 1) {
        const float c = (hx - ld_field<T>(d, copy, 3, o - Z)) - (hz - ld_field<T>(d, copy, 5, o - 1));
        st_field<T>(d, copy, 1, o, ld_field<T>(d, copy, 1, o) + ld_coef(d, 1, o) * c);
    }
    if (i >= 1 && j >= 1) {
        const float c = (hy - ld_field<T>(d, copy, 4, o - 1)) - (hx - ld_field<T>(d, copy, 3, o - P));
        st_field<T>(d, copy, 2, o, ld_field<T>(d, copy, 2, o) + ld_coef(d, 2, o) * c);
    }
}

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1216;   // 8 x 152 SMs; fixed so that the summation order is reproducible

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kRedThreads / 32; ++i) r += sh[i];
    return r;
}

// Reciprocal coefficients of the reductions as pairs (df.cuh): 1/ce (c = 0..2) and 1/ch (c = 3..5).
// Material-id mode keeps them in a shared table (filled by the block before use), scalar mode in six
// registers; per-position arrays take the reciprocal per cell (that mode is rare and slow anyway).
struct InvCoefDF {
    const CavityDesc *d;
    const df::F2 *tab;   // shared, 6 per id (COEF_ID8)
    df::F2 sc[6];        // COEF_SCALAR
    __device__ __forceinline__ df::F2 operator()(int c, long long o, int m) const {
        if (d->coef_mode == COEF_ID8) return tab[6 * m + c];
        if (d->coef_mode == COEF_SCALAR) return sc[c];
        return df::recip(d->coef[c][o]);
    }
};

// Fills tab (6 * ntab pairs, shared) and the scalar reciprocals; call with the whole block, then sync.
__device__ __forceinline__ InvCoefDF make_inv_coef_df(const CavityDesc &d, df::F2 *tab) {
    InvCoefDF r;
    r.d = &d;
    r.tab = tab;
    for (int c = 0; c < 3; ++c) {
        r.sc[c] = df::recip(d.ce[c]);
        r.sc[3 + c] = df::recip(d.ch[c]);
    }
    if (d.coef_mode == COEF_ID8)
        for (int e = threadIdx.x; e < 6 * d.ntab; e += blockDim.x) {
            const int m = e / 6, c = e % 6;
            tab[e] = df::recip(d.table[8 * m + (c < 3 ? c : c + 1)]);
        }
    return r;
}

// 1/ch at far-face entry fi of face array c, as a pair and in FP64.
__device__ __forceinline__ df::F2 face_inv_ch_df(const CavityDesc &d, int c, long long fi) {
    return df::recip(d.coef_mode == COEF_SCALAR ? d.ch[c] : d.face_ch[c][fi]);
}
__device__ __forceinline__ double face_inv_ch64(const CavityDesc &d, int c, long long fi) {
    return d.coef_mode == COEF_SCALAR ? 1.0 / (double)d.ch[c] : 1.0 / (double)d.face_ch[c][fi];
}

// Per block, in a fixed order (warps over rows, lanes along x; far-face H appended):
//   WHAT == 0: energy sum  E^2/ce + H^2/ch - H curl E   (W without the 1/2 dt/dx factor)
//   WHAT == 1: sum of divE^2 over interior nodes and of divH^2 over cells.
// Every term is formed from the stored values with error-free FP32 transformations (the curl
// differences as exact pairs, the reciprocal coefficients as pairs; df.cuh) and a lane accumulates
// its cells of a row with Dot2, about 2^-48 relative; the row sums are added in FP64, then per block
// and over blocks in a fixed order, so the result is deterministic.  (GB300's FP64 rate made the same
// sums in FP64 eight times slower at 512^3.)
template <typename T, int WHAT>
__global__ void __launch_bounds__(kRedThreads) reduce_kernel(const CavityDesc d, int copy, double *partial) {
    __shared__ double sh[kRedThreads / 32];
    __shared__ df::F2 itab[6 * kMaxTable];
    const int nx = d.nx, ny = d.ny;
    const long long P = d.pitch, Z = d.plane;
    double s0 = 0.0, s1 = 0.0;
    const bool ids = d.coef_mode == COEF_ID8;
    const InvCoefDF IC = make_inv_coef_df(d, itab);
    __syncthreads();
    const int nz = d.nz;
    auto F = [&](int f, long long o) -> float { return ld_field<T>(d, copy, f, o); };
    auto ICo = [&](int c, long long o) -> df::F2 { return IC(c, o, ids ? d.id[o] : 0); };
    // one warp per (j, k) row, lanes along x: coalesced loads
    const int lane = threadIdx.x & 31;
    // rows of the planes [kr_lo, kr_hi) (the owned cells of a z-slab; every plane otherwise)
    const long long nrows = (long long)ny * (d.kr_hi - d.kr_lo);
    const long long nwarps = ((long long)gridDim.x * kRedThreads) >> 5;
    for (long long r = ((long long)blockIdx.x * kRedThreads + threadIdx.x) >> 5; r < nrows; r += nwarps) {
        const int j = (int)(r % ny), k = d.kr_lo + (int)(r / ny);
        df::Acc a0, a1;
        for (int i = lane; i < nx; i += 32) {
            const long long o = (long long)k * Z + (long long)j * P + i;
            const float ex = F(0, o), ey = F(1, o), ez = F(2, o), hx = F(3, o), hy = F(4, o), hz = F(5, o);
            const int m = ids ? d.id[o] : 0;
            if (WHAT == 0) {
                const float ex_j1 = j + 1 < ny ? F(0, o + P) : 0.f, ex_k1 = k + 1 < nz ? F(0, o + Z) : 0.f;
                const float ey_i1 = i + 1 < nx ? F(1, o + 1) : 0.f, ey_k1 = k + 1 < nz ? F(1, o + Z) : 0.f;
                const float ez_i1 = i + 1 < nx ? F(2, o + 1) : 0.f, ez_j1 = j + 1 < ny ? F(2, o + P) : 0.f;
                a0.sq_times(ex, IC(0, o, m));
                a0.sq_times(ey, IC(1, o, m));
                a0.sq_times(ez, IC(2, o, m));
                a0.sq_times(hx, IC(3, o, m));
                a0.prod(-hx, df::diff2(ez_j1, ez, ey_k1, ey));
                a0.sq_times(hy, IC(4, o, m));
                a0.prod(-hy, df::diff2(ex_k1, ex, ez_i1, ez));
                a0.sq_times(hz, IC(5, o, m));
                a0.prod(-hz, df::diff2(ey_i1, ey, ex_j1, ex));
            } else {
                if (i >= 1 && j >= 1 && k >= 1) {
                    df::Acc de;   // sum over c of D_c(node) - D_c(node - e_c), D = E / ce
                    de.prod(ex, IC(0, o, m));
                    de.prod(-F(0, o - 1), ICo(0, o - 1));
                    de.prod(ey, IC(1, o, m));
                    de.prod(-F(1, o - P), ICo(1, o - P));
                    de.prod(ez, IC(2, o, m));
                    de.prod(-F(2, o - Z), ICo(2, o - Z));
                    a0.square(de.pair());
                }
                df::Acc dh;   // sum over c of B_c(cell + e_c) - B_c(cell), B = H / ch
                const long long fx = (long long)k * ny + j, fy = (long long)k * nx + i, fz = (long long)j * nx + i;
                if (i + 1 < nx) dh.prod(F(3, o + 1), ICo(3, o + 1));
                else dh.prod(d.face[0][fx], face_inv_ch_df(d, 0, fx));
                if (j + 1 < ny) dh.prod(F(4, o + P), ICo(4, o + P));
                else dh.prod(d.face[1][fy], face_inv_ch_df(d, 1, fy));
                if (k + 1 < nz) dh.prod(F(5, o + Z), ICo(5, o + Z));
                else dh.prod(d.face[2][fz], face_inv_ch_df(d, 2, fz));
                dh.prod(-hx, IC(3, o, m));
                dh.prod(-hy, IC(4, o, m));
                dh.prod(-hz, IC(5, o, m));
                a1.square(dh.pair());
            }
        }
        s0 += a0.take();
        s1 += a1.take();
    }
    if (WHAT == 0) {
        // constant far-face normal H: curl E vanishes there, so its energy term is H^2/ch (the x and y
        // faces over the summed planes, the z face when the range reaches it); few terms: FP64
        const int nk = d.kr_hi - d.kr_lo;
        const long long nfx = (long long)ny * nk, nfy = (long long)nx * nk, nfz = d.face_top ? (long long)nx * ny : 0;
        for (long long n = blockIdx.x * (long long)kRedThreads + threadIdx.x; n < nfx + nfy + nfz;
             n += (long long)gridDim.x * kRedThreads) {
            int c;
            long long fi;
            if (n < nfx) { c = 0; fi = n + (long long)d.kr_lo * ny; }
            else if (n < nfx + nfy) { c = 1; fi = n - nfx + (long long)d.kr_lo * nx; }
            else { c = 2; fi = n - nfx - nfy; }
            const double h = d.face[c][fi];
            s0 += h * h * face_inv_ch64(d, c, fi);
        }
    }
    const double a = block_sum(s0, sh);
    const double b = block_sum(s1, sh);
    if (threadIdx.x == 0) {
        partial[3 * blockIdx.x + 0] = WHAT == 0 ? a : 0.0;
        partial[3 * blockIdx.x + 1] = WHAT == 1 ? a : 0.0;
        partial[3 * blockIdx.x + 2] = b;
    }
}

__global__ void __launch_bounds__(kRedThreads) reduce_final_kernel(const double *partial, int nblocks, double *out) {
    __shared__ double sh[kRedThreads / 32];
    for (int q = 0; q < 3; ++q) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += kRedThreads) v += partial[3 * b + q];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) out[q] = v;
    }
}

template <typename T>
cudaError_t simple_step_typed(const CavityDesc &d, int copy, cudaStream_t s) {
    dim3 blk(BXs, BYs), grd((d.nx + BXs - 1) / BXs, (d.ny + BYs - 1) / BYs, d.nz);
    simple_h_kernel<T><<<grd, blk, 0, s>>>(d, copy);
    simple_e_kernel<T><<<grd, blk, 0, s>>>(d, copy);
    return cudaGetLastError();
}

#define FDTD_STORAGE_DISPATCH(storage, ...)                 \
    do {                                                     \
        if (storage == 0) { using T = float; __VA_ARGS__; }         \
        else if (storage == 1) { using T = __half; __VA_ARGS__; }   \
        else { using T = __nv_bfloat16; __VA_ARGS__; }              \
    } while (0)

}  // namespace

cudaError_t launch_pack(int storage, const CavityDesc &d, int copy, int comp, const float *canon, float *face,
                        cudaStream_t s) {
    dim3 blk(BXs, BYs), grd((d.nx + 1 + BXs - 1) / BXs, (d.ny + 1 + BYs - 1) / BYs, (d.nz + 1 + KZs - 1) / KZs);
    FDTD_STORAGE_DISPATCH(storage, pack_kernel<T><<<grd, blk, 0, s>>>(d, copy, comp, canon, face));
    return cudaGetLastError();
}

cudaError_t launch_unpack(int storage, const CavityDesc &d, int copy, int comp, float *canon, cudaStream_t s) {
    dim3 blk(BXs, BYs), grd((d.nx + 1 + BXs - 1) / BXs, (d.ny + 1 + BYs - 1) / BYs, (d.nz + 1 + KZs - 1) / KZs);
    FDTD_STORAGE_DISPATCH(storage, unpack_kernel<T><<<grd, blk, 0, s>>>(d, copy, comp, canon));
    return cudaGetLastError();
}

cudaError_t launch_maxabs(const float *canon, int comp, int nx, int ny, int nz, unsigned *out, cudaStream_t s) {
    dim3 blk(BXs, BYs), grd((nx + 1 + BXs - 1) / BXs, (ny + 1 + BYs - 1) / BYs, nz + 1);
    maxabs_kernel<<<grd, blk, 0, s>>>(canon, comp, nx, ny, nz, out);
    return cudaGetLastError();
}

cudaError_t launch_simple_step(int storage, const CavityDesc &d, int copy, cudaStream_t s) {
    cudaError_t e;
    FDTD_STORAGE_DISPATCH(storage, e = simple_step_typed<T>(d, copy, s));
    return e;
}

int reduction_blocks() { return kRedBlocks; }

cudaError_t launch_reductions(int storage, const CavityDesc &d, int copy, int what, double *partial, int nblocks,
                              double *out, cudaStream_t s, int order) {
    if (order == 4) {
        cudaError_t e = launch_reductions4(storage, d, copy, what, partial, nblocks, s);
        if (e != cudaSuccess) return e;
    } else if (what == 0)
        FDTD_STORAGE_DISPATCH(storage, reduce_kernel<T, 0><<<nblocks, kRedThreads, 0, s>>>(d, copy, partial));
    else
        FDTD_STORAGE_DISPATCH(storage, reduce_kernel<T, 1><<<nblocks, kRedThreads, 0, s>>>(d, copy, partial));
    reduce_final_kernel<<<1, kRedThreads, 0, s>>>(partial, nblocks, out);
    return cudaGetLastError();
}

}  // namespace fdtd
