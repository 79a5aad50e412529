// Fourth-order (2,4) Yee step, unfused (one thread per cell, two launches per step), and the FP64
// energy and divergence reductions of that scheme.
//
// The step is that of Eq. 2 with every difference replaced by the staggered fourth-order
// difference of order4.cuh (image-closed PEC walls).  Like the second-order unfused step it
// updates one copy of the fields in place (H from E, then E from H) and serves every coefficient
// mode, including per-position arrays; it is also the reference the fused fourth-order kernel
// is checked against bit for bit.
#include "df.cuh"
#include "launch.h"
#include "order4.cuh"

namespace fdtd {

namespace {

using namespace o4;

constexpr int BX4 = 32, BY4 = 8;

// H^{n+1/2} = H^{n-1/2} - ch curl4 E^n.  A tap outside [0, n) along its axis reads 0 (E at index n
// is tangential, hence 0; one past that is an image folded into the weights).
template <typename T>
__global__ void simple4_h_kernel(const CavityDesc d, int copy) {
    const int i = blockIdx.x * BX4 + threadIdx.x, j = blockIdx.y * BY4 + threadIdx.y, k = blockIdx.z;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    if (i >= nx || j >= ny) return;
    const long long P = d.pitch, Z = d.plane;
    const long long o = (long long)k * Z + (long long)j * P + i;
    auto E = [&](int f, int di, int dj, int dk) -> float {
        const int a = i + di, b = j + dj, c = k + dk;
        if (a < 0 || a >= nx || b < 0 || b >= ny || c < 0 || c >= nz) return 0.f;
        return ld_field<T>(d, copy, f, o + dk * Z + dj * P + di);
    };
    const float wax = wa_h(i, nx), wbx = wb_h(i, nx), way = wa_h(j, ny), wby = wb_h(j, ny);
    const float waz = wa_h(k, nz), wbz = wb_h(k, nz);
    const float dyEz = d4(E(2, 0, -1, 0), E(2, 0, 0, 0), E(2, 0, 1, 0), E(2, 0, 2, 0), way, wby);
    const float dzEy = d4(E(1, 0, 0, -1), E(1, 0, 0, 0), E(1, 0, 0, 1), E(1, 0, 0, 2), waz, wbz);
    const float dzEx = d4(E(0, 0, 0, -1), E(0, 0, 0, 0), E(0, 0, 0, 1), E(0, 0, 0, 2), waz, wbz);
    const float dxEz = d4(E(2, -1, 0, 0), E(2, 0, 0, 0), E(2, 1, 0, 0), E(2, 2, 0, 0), wax, wbx);
    const float dxEy = d4(E(1, -1, 0, 0), E(1, 0, 0, 0), E(1, 1, 0, 0), E(1, 2, 0, 0), wax, wbx);
    const float dyEx = d4(E(0, 0, -1, 0), E(0, 0, 0, 0), E(0, 0, 1, 0), E(0, 0, 2, 0), way, wby);
    // each bracket is -(curl E): H + ch * bracket
    st_field<T>(d, copy, 3, o, __fmaf_rn(ld_coef(d, 3, o), __fsub_rn(dzEy, dyEz), ld_field<T>(d, copy, 3, o)));
    st_field<T>(d, copy, 4, o, __fmaf_rn(ld_coef(d, 4, o), __fsub_rn(dxEz, dzEx), ld_field<T>(d, copy, 4, o)));
    st_field<T>(d, copy, 5, o, __fmaf_rn(ld_coef(d, 5, o), __fsub_rn(dyEx, dxEy), ld_field<T>(d, copy, 5, o)));
}

// E^{n+1} = E^n + ce curl4 H^{n+1/2} on entries not tangential to a face.  H taps outside [0, n)
// read 0 (images folded into the weights).
template <typename T>
__global__ void simple4_e_kernel(const CavityDesc d, int copy) {
    const int i = blockIdx.x * BX4 + threadIdx.x, j = blockIdx.y * BY4 + threadIdx.y, k = blockIdx.z;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    if (i >= nx || j >= ny) return;
    const long long P = d.pitch, Z = d.plane;
    const long long o = (long long)k * Z + (long long)j * P + i;
    auto H = [&](int f, int di, int dj, int dk) -> float {
        const int a = i + di, b = j + dj, c = k + dk;
        if (a < 0 || a >= nx || b < 0 || b >= ny || c < 0 || c >= nz) return 0.f;
        return ld_field<T>(d, copy, f, o + dk * Z + dj * P + di);
    };
    const float wax = wa_e(i, nx), wbx = wb_e(i, nx), way = wa_e(j, ny), wby = wb_e(j, ny);
    const float waz = wa_e(k, nz), wbz = wb_e(k, nz);
    if (j >= 1 && k >= 1) {
        const float dyHz = d4(H(5, 0, -2, 0), H(5, 0, -1, 0), H(5, 0, 0, 0), H(5, 0, 1, 0), way, wby);
        const float dzHy = d4(H(4, 0, 0, -2), H(4, 0, 0, -1), H(4, 0, 0, 0), H(4, 0, 0, 1), waz, wbz);
        st_field<T>(d, copy, 0, o, __fmaf_rn(ld_coef(d, 0, o), __fsub_rn(dyHz, dzHy), ld_field<T>(d, copy, 0, o)));
    }
    if (i >= 1 && k >= 1) {
        const float dzHx = d4(H(3, 0, 0, -2), H(3, 0, 0, -1), H(3, 0, 0, 0), H(3, 0, 0, 1), waz, wbz);
        const float dxHz = d4(H(5, -2, 0, 0), H(5, -1, 0, 0), H(5, 0, 0, 0), H(5, 1, 0, 0), wax, wbx);
        st_field<T>(d, copy, 1, o, __fmaf_rn(ld_coef(d, 1, o), __fsub_rn(dzHx, dxHz), ld_field<T>(d, copy, 1, o)));
    }
    if (i >= 1 && j >= 1) {
        const float dxHy = d4(H(4, -2, 0, 0), H(4, -1, 0, 0), H(4, 0, 0, 0), H(4, 1, 0, 0), wax, wbx);
        const float dyHx = d4(H(3, 0, -2, 0), H(3, 0, -1, 0), H(3, 0, 0, 0), H(3, 0, 1, 0), way, wby);
        st_field<T>(d, copy, 2, o, __fmaf_rn(ld_coef(d, 2, o), __fsub_rn(dxHy, dyHx), ld_field<T>(d, copy, 2, o)));
    }
}

constexpr int kRed4Threads = 256;

// Terms of the fourth-order differences for the compensated reductions (df.cuh), with the step's own
// weights (the FP32 values of c1, c2 and c1 + c2 the kernels use): the invariants of the discrete
// scheme that is actually stepped.  acc += sign (c2 (b2 - a2) + wb b - wa a).
__device__ __forceinline__ void d4_acc(df::Acc &acc, float sign, float a2, float a, float b, float b2, float wa,
                                       float wb) {
    acc.prod(sign * kC2, b2);
    acc.prod(-sign * kC2, a2);
    acc.prod(sign * wb, b);
    acc.prod(-sign * wa, a);
}
// The same with taps given as pairs (D = E / ce, B = H / ch).
__device__ __forceinline__ void d4_acc(df::Acc &acc, df::F2 a2, df::F2 a, df::F2 b, df::F2 b2, float wa, float wb) {
    acc.prod(kC2, b2);
    acc.prod(-kC2, a2);
    acc.prod(wb, b);
    acc.prod(-wa, a);
}

__device__ __forceinline__ double block_sum4(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < kRed4Threads / 32; ++q) r += sh[q];
    return r;
}

// Per block, one warp per (j, k) row, lanes along x:
//   WHAT == 0: sum  E^2/ce + H^2/ch - H curl4 E  (W without the 1/2 dt/dx factor), far-face H appended;
//   WHAT == 1: sum of div4E^2 over interior nodes and of div4B^2 over cells, B = H/ch, with D = E/ce
//   mirrored evenly and B oddly past a wall (the same folded weights as the step; B at index n is the
//   constant far-face H).
// Every term is formed with error-free FP32 transformations and a lane accumulates its cells of a row
// with Dot2 (about 2^-48 relative, df.cuh); row sums are added in FP64 in a fixed order.
template <typename T, int WHAT>
__global__ void __launch_bounds__(kRed4Threads) reduce4_kernel(const CavityDesc d, int copy, double *partial) {
    __shared__ double sh[kRed4Threads / 32];
    __shared__ df::F2 itab[6 * kMaxTable];   // 1/ce xyz, 1/ch xyz per material id
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const long long P = d.pitch, Z = d.plane;
    double s0 = 0.0, s1 = 0.0;
    df::F2 isc[6];
    for (int c = 0; c < 3; ++c) {
        isc[c] = df::recip(d.ce[c]);
        isc[3 + c] = df::recip(d.ch[c]);
    }
    if (d.coef_mode == COEF_ID8)
        for (int e = threadIdx.x; e < 6 * d.ntab; e += kRed4Threads) {
            const int m = e / 6, c = e % 6;
            itab[e] = df::recip(d.table[8 * m + (c < 3 ? c : c + 1)]);
        }
    __syncthreads();
    auto IC = [&](int c, long long o) -> df::F2 {
        if (d.coef_mode == COEF_ID8) return itab[6 * d.id[o] + c];
        if (d.coef_mode == COEF_SCALAR) return isc[c];
        return df::recip(d.coef[c][o]);
    };
    auto face_inv_ch = [&](int c, long long fi) -> df::F2 {
        return d.coef_mode == COEF_SCALAR ? isc[3 + c] : df::recip(d.face_ch[c][fi]);
    };
    const df::F2 zero{0.f, 0.f};
    const int lane = threadIdx.x & 31;
    // rows of the planes [kr_lo, kr_hi) (the owned cells of a z-slab; every plane otherwise)
    const long long nrows = (long long)ny * (d.kr_hi - d.kr_lo);
    const long long nwarps = ((long long)gridDim.x * kRed4Threads) >> 5;
    for (long long r = ((long long)blockIdx.x * kRed4Threads + threadIdx.x) >> 5; r < nrows; r += nwarps) {
        const int j = (int)(r % ny), k = d.kr_lo + (int)(r / ny);
        df::Acc a0, a1;
        for (int i = lane; i < nx; i += 32) {
            const long long o = (long long)k * Z + (long long)j * P + i;
            auto F = [&](int f, int di, int dj, int dk) -> float {   // 0 outside the active range
                const int a = i + di, b = j + dj, c = k + dk;
                if (a < 0 || a >= nx || b < 0 || b >= ny || c < 0 || c >= nz) return 0.f;
                return ld_field<T>(d, copy, f, o + dk * Z + dj * P + di);
            };
            if (WHAT == 0) {
                const float wax = wa_h(i, nx), wbx = wb_h(i, nx), way = wa_h(j, ny), wby = wb_h(j, ny);
                const float waz = wa_h(k, nz), wbz = wb_h(k, nz);
                df::Acc cx, cy, cz;   // the three curl components as pairs
                d4_acc(cx, 1.f, F(2, 0, -1, 0), F(2, 0, 0, 0), F(2, 0, 1, 0), F(2, 0, 2, 0), way, wby);
                d4_acc(cx, -1.f, F(1, 0, 0, -1), F(1, 0, 0, 0), F(1, 0, 0, 1), F(1, 0, 0, 2), waz, wbz);
                d4_acc(cy, 1.f, F(0, 0, 0, -1), F(0, 0, 0, 0), F(0, 0, 0, 1), F(0, 0, 0, 2), waz, wbz);
                d4_acc(cy, -1.f, F(2, -1, 0, 0), F(2, 0, 0, 0), F(2, 1, 0, 0), F(2, 2, 0, 0), wax, wbx);
                d4_acc(cz, 1.f, F(1, -1, 0, 0), F(1, 0, 0, 0), F(1, 1, 0, 0), F(1, 2, 0, 0), wax, wbx);
                d4_acc(cz, -1.f, F(0, 0, -1, 0), F(0, 0, 0, 0), F(0, 0, 1, 0), F(0, 0, 2, 0), way, wby);
                const float ex = F(0, 0, 0, 0), ey = F(1, 0, 0, 0), ez = F(2, 0, 0, 0);
                const float hx = F(3, 0, 0, 0), hy = F(4, 0, 0, 0), hz = F(5, 0, 0, 0);
                a0.sq_times(ex, IC(0, o));
                a0.sq_times(ey, IC(1, o));
                a0.sq_times(ez, IC(2, o));
                a0.sq_times(hx, IC(3, o));
                a0.prod(-hx, cx.pair());
                a0.sq_times(hy, IC(4, o));
                a0.prod(-hy, cy.pair());
                a0.sq_times(hz, IC(5, o));
                a0.prod(-hz, cz.pair());
            } else {
                if (i >= 1 && j >= 1 && k >= 1) {
                    // D_a = E_a / ce_a; taps at E index -1 or n along a read 0 (folded even images)
                    auto D = [&](int f, int di, int dj, int dk) -> df::F2 {
                        const int a = i + di, b = j + dj, c = k + dk;
                        if (a < 0 || a >= nx || b < 0 || b >= ny || c < 0 || c >= nz) return zero;
                        const long long q = o + dk * Z + dj * P + di;
                        return df::mul(ld_field<T>(d, copy, f, q), IC(f, q));
                    };
                    df::Acc de;
                    d4_acc(de, D(0, -2, 0, 0), D(0, -1, 0, 0), D(0, 0, 0, 0), D(0, 1, 0, 0), wa_e(i, nx), wb_e(i, nx));
                    d4_acc(de, D(1, 0, -2, 0), D(1, 0, -1, 0), D(1, 0, 0, 0), D(1, 0, 1, 0), wa_e(j, ny), wb_e(j, ny));
                    d4_acc(de, D(2, 0, 0, -2), D(2, 0, 0, -1), D(2, 0, 0, 0), D(2, 0, 0, 1), wa_e(k, nz), wb_e(k, nz));
                    a0.square(de.pair());
                }
                // B_a = H_a / ch_a at a node index along a: index n is the far face, beyond it 0
                auto Bx = [&](int di) -> df::F2 {
                    const int a = i + di;
                    if (a < 0 || a > nx) return zero;
                    if (a == nx) {
                        const long long fi = (long long)k * ny + j;
                        return df::mul(d.face[0][fi], face_inv_ch(0, fi));
                    }
                    return df::mul(ld_field<T>(d, copy, 3, o + di), IC(3, o + di));
                };
                auto By = [&](int dj) -> df::F2 {
                    const int b = j + dj;
                    if (b < 0 || b > ny) return zero;
                    if (b == ny) {
                        const long long fi = (long long)k * nx + i;
                        return df::mul(d.face[1][fi], face_inv_ch(1, fi));
                    }
                    return df::mul(ld_field<T>(d, copy, 4, o + dj * P), IC(4, o + dj * P));
                };
                auto Bz = [&](int dk) -> df::F2 {
                    const int c = k + dk;
                    if (c < 0 || c > nz) return zero;
                    if (c == nz) {
                        const long long fi = (long long)j * nx + i;
                        return df::mul(d.face[2][fi], face_inv_ch(2, fi));
                    }
                    return df::mul(ld_field<T>(d, copy, 5, o + dk * Z), IC(5, o + dk * Z));
                };
                // the image of B one past a wall is odd: the folded weights of a difference of E
                df::Acc dh;
                d4_acc(dh, Bx(-1), Bx(0), Bx(1), Bx(2), wa_h(i, nx), wb_h(i, nx));
                d4_acc(dh, By(-1), By(0), By(1), By(2), wa_h(j, ny), wb_h(j, ny));
                d4_acc(dh, Bz(-1), Bz(0), Bz(1), Bz(2), wa_h(k, nz), wb_h(k, nz));
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
        for (long long n = blockIdx.x * (long long)kRed4Threads + threadIdx.x; n < nfx + nfy + nfz;
             n += (long long)gridDim.x * kRed4Threads) {
            int c;
            long long fi;
            if (n < nfx) { c = 0; fi = n + (long long)d.kr_lo * ny; }
            else if (n < nfx + nfy) { c = 1; fi = n - nfx + (long long)d.kr_lo * nx; }
            else { c = 2; fi = n - nfx - nfy; }
            const double h = d.face[c][fi];
            const double ich = d.coef_mode == COEF_SCALAR ? 1.0 / (double)d.ch[c] : 1.0 / (double)d.face_ch[c][fi];
            s0 += h * h * ich;
        }
    }
    const double a = block_sum4(s0, sh);
    const double b = block_sum4(s1, sh);
    if (threadIdx.x == 0) {
        partial[3 * blockIdx.x + 0] = WHAT == 0 ? a : 0.0;
        partial[3 * blockIdx.x + 1] = WHAT == 1 ? a : 0.0;
        partial[3 * blockIdx.x + 2] = b;
    }
}

template <typename T>
cudaError_t simple4_step_typed(const CavityDesc &d, int copy, cudaStream_t s) {
    dim3 blk(BX4, BY4), grd((d.nx + BX4 - 1) / BX4, (d.ny + BY4 - 1) / BY4, d.nz);
    simple4_h_kernel<T><<<grd, blk, 0, s>>>(d, copy);
    simple4_e_kernel<T><<<grd, blk, 0, s>>>(d, copy);
    return cudaGetLastError();
}

#define FDTD4_STORAGE_DISPATCH(storage, ...)                        \
    do {                                                            \
        if (storage == 0) { using T = float; __VA_ARGS__; }         \
        else if (storage == 1) { using T = __half; __VA_ARGS__; }   \
        else { using T = __nv_bfloat16; __VA_ARGS__; }              \
    } while (0)

}  // namespace

cudaError_t launch_simple4_step(int storage, const CavityDesc &d, int copy, cudaStream_t s) {
    cudaError_t e;
    FDTD4_STORAGE_DISPATCH(storage, e = simple4_step_typed<T>(d, copy, s));
    return e;
}

cudaError_t launch_reductions4(int storage, const CavityDesc &d, int copy, int what, double *partial, int nblocks,
                               cudaStream_t s) {
    if (what == 0)
        FDTD4_STORAGE_DISPATCH(storage, reduce4_kernel<T, 0><<<nblocks, kRed4Threads, 0, s>>>(d, copy, partial));
    else
        FDTD4_STORAGE_DISPATCH(storage, reduce4_kernel<T, 1><<<nblocks, kRed4Threads, 0, s>>>(d, copy, partial));
    return cudaGetLastError();
}

}  // namespace fdtd
