// Generic kernels: any order N, any storage precision.
//
//  * k_substep_generic   one thread per cell; for every target of the class, gathers its <= 10
//                        partners through the partner table (Section 3.2's unrolled sparse
//                        product, here table driven) and applies the exact substep of Eq. (5).
//  * k_media_factors     FP64 per-cell substep factors at the staggered points (Section 3.2:
//                        parameters stored per cell, interpolated to the sub-grids).
//  * conversions, the FP64 sum of u_0 and the non-finite count.
#include <cuda_bf16.h>

#include "rtpn_internal.h"

namespace rtpn {

// ------------------------------------------------------------------ storage <-> math helpers
template <typename S, typename F>
__device__ __forceinline__ F ld(const S* p) { return static_cast<F>(*p); }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16, float>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <typename S, typename F>
__device__ __forceinline__ void st(S* p, F v) { *p = static_cast<S>(v); }
template <>
__device__ __forceinline__ void st<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
}

__device__ __forceinline__ long long cell_index(const Geom& g, int x, int y, int z) {
    return ((long long)z * g.ny + y) * g.nx + x;
}

// neighbour along axis (0 x, 1 y, 2 z) in direction dir (+1/-1); false if outside (vacuum)
__device__ __forceinline__ bool neighbour(const Geom& g, int x, int y, int z, int axis, int dir,
                                          long long* idx) {
    int c[3] = {x, y, z};
    const int n[3] = {g.nx, g.ny, g.nz};
    int v = c[axis] + dir;
    if (v < 0 || v >= n[axis]) {
        if (g.bc != RTPN_BC_PERIODIC) return false;
        v = v < 0 ? v + n[axis] : v - n[axis];
    }
    c[axis] = v;
    *idx = cell_index(g, c[0], c[1], c[2]);
    return true;
}

// ------------------------------------------------------------------ substep (generic gather)
template <typename S, typename F>
__global__ void k_substep_generic(S* __restrict__ u, const F* __restrict__ fac,
                                  PartnerTable<F> tab, Geom g, int fac_ofs) {
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= g.V) return;
    const int x = (int)(cell % g.nx);
    const int y = (int)((cell / g.nx) % g.ny);
    const int z = (int)(cell / ((long long)g.nx * g.ny));
    // neighbour offsets: code = axis*2 + (upper ? 1 : 0)
    long long nb[6];
    bool ok[6];
    for (int code = 0; code < 6; ++code) {
        ok[code] = neighbour(g, x, y, z, code >> 1, (code & 1) ? 1 : -1, &nb[code]);
        if (!ok[code]) nb[code] = cell;
    }
    for (int t = 0; t < tab.na; ++t) {
        F r = F(0);
        for (int p = tab.row[t]; p < tab.row[t + 1]; ++p) {
            const S* ub = u + (long long)tab.src[p] * g.V;
            const int code = tab.code[p];
            const F centre = ld<S, F>(ub + cell);
            const F other = ok[code] ? ld<S, F>(ub + nb[code]) : F(0);
            // r = q - sum coef * D u ; coef carries 1/h and the sign of the difference direction
            r -= tab.coef[p] * (other - centre);
        }
        const int fp = tab.fplane[t];
        S* ua = u + (long long)(tab.a0 + t) * g.V + cell;
        const F old = ld<S, F>(ua);
        F nv;
        if (fp == FAC_U0) {
            const F al = fac[(long long)FAC_U0 * g.V + cell];
            const F be = fac[(long long)(FAC_U0 + 1) * g.V + cell];
            const F ga = fac[(long long)(FAC_U0 + 2) * g.V + cell];
            nv = al * old + be * r + ga;
        } else {
            const F al = fac[(long long)(fp + fac_ofs) * g.V + cell];
            const F be = fac[(long long)(fp + fac_ofs + 1) * g.V + cell];
            nv = al * old + be * r;
        }
        st<S, F>(ua, nv);
    }
}

template <typename S, typename F>
void launch_substep_generic(S* u, const F* fac, const PartnerTable<F>& tab, const Geom& g,
                            int fac_ofs, cudaStream_t stream) {
    const int bs = 256;
    const long long nb = (g.V + bs - 1) / bs;
    k_substep_generic<S, F><<<(unsigned)nb, bs, 0, stream>>>(u, fac, tab, g, fac_ofs);
}

template void launch_substep_generic<double, double>(double*, const double*,
                                                     const PartnerTable<double>&, const Geom&, int,
                                                     cudaStream_t);
template void launch_substep_generic<float, float>(float*, const float*, const PartnerTable<float>&,
                                                   const Geom&, int, cudaStream_t);
template void launch_substep_generic<__nv_bfloat16, float>(__nv_bfloat16*, const float*,
                                                           const PartnerTable<float>&, const Geom&,
                                                           int, cudaStream_t);

// ------------------------------------------------------------------ media -> substep factors
// alpha = exp(-c tau), beta = tau E(-c tau) = -expm1(-c tau)/c (beta = tau at c = 0), for any real c
// (the same analytic expression on both sides of 0, so a derivative in sigma taken by differences
// at sigma = 0 sees one smooth function); FP64 library exp/expm1, rounded to F on store.
__device__ __forceinline__ void factors(double c, double tau, double* al, double* be) {
    *al = exp(-c * tau);
    *be = c != 0.0 ? -expm1(-c * tau) / c : tau;
}

template <typename F>
__global__ void k_media_factors(const double* __restrict__ sa, const double* __restrict__ ss,
                                const double* __restrict__ q, F* __restrict__ fac, Geom g,
                                double dt, const double* __restrict__ scat, int N) {
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= g.V) return;
    const int x = (int)(cell % g.nx);
    const int y = (int)((cell / g.nx) % g.ny);
    const int z = (int)(cell / ((long long)g.nx * g.ny));
    for (int code = 0; code < 8; ++code) {
        const int gx = code & 1, gy = (code >> 1) & 1, gz = (code >> 2) & 1;
        // mean of sigma_a + sigma_s over the cells adjacent to the staggered point: cell + {0,1}
        // along every axis whose slot is 2 (periodic: wrapped; vacuum: in-domain cells only)
        double sum = 0.0, sum_a = 0.0, sum_s = 0.0;
        int cnt = 0;
        for (int dz = 0; dz <= gz; ++dz)
            for (int dy = 0; dy <= gy; ++dy)
                for (int dx = 0; dx <= gx; ++dx) {
                    int xx = x + dx, yy = y + dy, zz = z + dz;
                    if (xx >= g.nx || yy >= g.ny || zz >= g.nz) {
                        if (g.bc != RTPN_BC_PERIODIC) continue;
                        if (xx >= g.nx) xx -= g.nx;
                        if (yy >= g.ny) yy -= g.ny;
                        if (zz >= g.nz) zz -= g.nz;
                    }
                    const long long j = cell_index(g, xx, yy, zz);
                    sum += sa[j] + ss[j];
                    sum_a += sa[j];
                    sum_s += ss[j];
                    ++cnt;
                }
        if (scat) {
            // orders l >= 1 of the slot's class (an even count of 2-slots: even l), Section 2's
            // Sigma_tl = sigma_a + (1 - f_l) sigma_s from the point means
            const int cls = (gx + gy + gz) & 1;
            for (int l = cls == 0 ? 2 : 1; l <= N; l += 2) {
                const double cl = (sum_a + (1.0 - scat[l]) * sum_s) / cnt;
                double al, be;
                factors(cl, dt, &al, &be);
                const int p = aniso_plane(N, code, l);
                fac[(long long)p * g.V + cell] = (F)al;
                fac[(long long)(p + 1) * g.V + cell] = (F)be;
                factors(cl, 0.5 * dt, &al, &be);
                fac[(long long)(p + aniso_half_ofs(N)) * g.V + cell] = (F)al;
                fac[(long long)(p + aniso_half_ofs(N) + 1) * g.V + cell] = (F)be;
            }
        }
        const double c = sum / cnt;
        double al, be;
        factors(c, dt, &al, &be);
        fac[(long long)(FAC_FULL + 2 * code) * g.V + cell] = (F)al;
        fac[(long long)(FAC_FULL + 2 * code + 1) * g.V + cell] = (F)be;
        factors(c, 0.5 * dt, &al, &be);
        fac[(long long)(FAC_HALF + 2 * code) * g.V + cell] = (F)al;
        fac[(long long)(FAC_HALF + 2 * code + 1) * g.V + cell] = (F)be;
    }
    double al, be;
    factors(sa[cell], dt, &al, &be);
    fac[(long long)FAC_U0 * g.V + cell] = (F)al;
    fac[(long long)(FAC_U0 + 1) * g.V + cell] = (F)be;
    fac[(long long)(FAC_U0 + 2) * g.V + cell] = (F)(be * q[cell]);
}

template <typename F>
void launch_media_factors(const double* sa, const double* ss, const double* q, F* fac,
                          const Geom& g, double dt, const double* scat, int N, cudaStream_t stream) {
    const int bs = 256;
    const long long nb = (g.V + bs - 1) / bs;
    k_media_factors<F><<<(unsigned)nb, bs, 0, stream>>>(sa, ss, q, fac, g, dt, scat, N);
}
template void launch_media_factors<double>(const double*, const double*, const double*, double*,
                                           const Geom&, double, const double*, int, cudaStream_t);
template void launch_media_factors<float>(const double*, const double*, const double*, float*,
                                          const Geom&, double, const double*, int, cudaStream_t);

// ------------------------------------------------------------------ conversions
template <typename A, typename B>
__device__ __forceinline__ B conv(A v) { return static_cast<B>(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 conv<double, __nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 conv<float, __nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ double conv<__nv_bfloat16, double>(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
}
template <>
__device__ __forceinline__ float conv<__nv_bfloat16, float>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = conv<A, B>(in[i]);
}

template <typename Sin, typename Sout>
void launch_convert(const Sin* in, Sout* out, long long n, cudaStream_t stream) {
    if (n <= 0) return;
    const int bs = 256;
    long long nb = (n + bs - 1) / bs;
    if (nb > 152 * 64) nb = 152 * 64;
    k_convert<Sin, Sout><<<(unsigned)nb, bs, 0, stream>>>(in, out, n);
}
#define RTPN_CONV(A, B) template void launch_convert<A, B>(const A*, B*, long long, cudaStream_t);
RTPN_CONV(double, double)
RTPN_CONV(double, float)
RTPN_CONV(double, __nv_bfloat16)
RTPN_CONV(float, double)
RTPN_CONV(float, float)
RTPN_CONV(float, __nv_bfloat16)
RTPN_CONV(__nv_bfloat16, double)
RTPN_CONV(__nv_bfloat16, float)
#undef RTPN_CONV

// ------------------------------------------------------------------ FP64 reductions
template <typename S>
__device__ __forceinline__ double as_double(S v) { return (double)v; }
template <>
__device__ __forceinline__ double as_double<__nv_bfloat16>(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
}

// Fixed grid and fixed per-thread order: bitwise reproducible.
template <typename S>
__global__ void k_sum_partial(const S* __restrict__ x, long long n, double* __restrict__ partial) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc += as_double(x[i]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) partial[blockIdx.x] = acc;
    }
}

__global__ void k_sum_final(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) *out = acc;
    }
}

template <typename S>
void launch_sum(const S* x, long long n, double* partial, int nblocks, double* out,
                cudaStream_t stream) {
    k_sum_partial<S><<<nblocks, 256, 0, stream>>>(x, n, partial);
    k_sum_final<<<1, 1024, 0, stream>>>(partial, nblocks, out);
}
template void launch_sum<double>(const double*, long long, double*, int, double*, cudaStream_t);
template void launch_sum<float>(const float*, long long, double*, int, double*, cudaStream_t);
template void launch_sum<__nv_bfloat16>(const __nv_bfloat16*, long long, double*, int, double*,
                                        cudaStream_t);

template <typename S>
__global__ void k_count_nonfinite(const S* __restrict__ x, long long n,
                                  unsigned long long* __restrict__ out) {
    unsigned long long c = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        c += isfinite(as_double(x[i])) ? 0ull : 1ull;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

template <typename S>
void launch_count_nonfinite(const S* x, long long n, unsigned long long* out, cudaStream_t stream) {
    cudaMemsetAsync(out, 0, sizeof(unsigned long long), stream);
    k_count_nonfinite<S><<<152 * 8, 256, 0, stream>>>(x, n, out);
}
template void launch_count_nonfinite<double>(const double*, long long, unsigned long long*,
                                             cudaStream_t);
template void launch_count_nonfinite<float>(const float*, long long, unsigned long long*,
                                            cudaStream_t);
template void launch_count_nonfinite<__nv_bfloat16>(const __nv_bfloat16*, long long,
                                                    unsigned long long*, cudaStream_t);

}  // namespace rtpn
