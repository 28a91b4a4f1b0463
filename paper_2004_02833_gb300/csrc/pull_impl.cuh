// The staged adjoint's per-cell arithmetic, __host__ __device__ so that a host program can run it
// over bounds-checked memory when checking it: the factor derivatives of Eq. (5) and the pull-back
// through one pass from its stored pre- and post-pass states.
#pragma once

#include <map>
#include <vector>

#include "window_impl.cuh"  // RTPN_HD, RTPN_CHECK_PTR, rtpn_internal.h

namespace rtpn {
namespace adj {

// E'(x) for E(x) = expm1(x) / x of Eq. (5).  For |x| < 1 its Taylor polynomial
// sum_{k<24} (k+1)/(k+2)! x^k by Horner's rule (coefficients built from the recurrence
// c_k = c_{k-1} (k+1) / (k (k+2)), c_0 = 1/2; the tail is below 1e-23); for |x| >= 1 the form
// (x e^x - expm1(x)) / x^2, whose numerator no longer cancels.  The closed form near 0 would lose
// about eps / x^2 of its value (1e-10 at |x| = 1e-3).
RTPN_HD double dE(double x) {
    if (fabs(x) < 1.0) {
        constexpr int K = 24;
        double c[K];
        c[0] = 0.5;
#pragma unroll
        for (int k = 1; k < K; ++k) c[k] = c[k - 1] * (double)(k + 1) / ((double)k * (double)(k + 2));
        double p = c[K - 1];
#pragma unroll
        for (int k = K - 2; k >= 0; --k) p = fma(p, x, c[k]);
        return p;
    }
    return (x * exp(x) - expm1(x)) / (x * x);
}

// dalpha/dc and dbeta/dc per slot code for tau = dt (planes 0..15) and dt/2 (16..31), u_0 (32, 33)
constexpr int DFAC_PLANES = 34;

// The factor derivatives of one cell: dalpha/dc = -tau alpha, dbeta/dc = -tau^2 E'(-c tau) at c,
// the mean of sigma_a + sigma_s over the cells adjacent to each sub-grid point (sigma_a for u_0).
template <typename F>
RTPN_HD void factor_derivatives(const double* sa, const double* ss, F* dfac, const Geom& g, double dt,
                                long long cell) {
    const int x = (int)(cell % g.nx), y = (int)((cell / g.nx) % g.ny), z = (int)(cell / ((long long)g.nx * g.ny));
    for (int code = 0; code < 8; ++code) {
        const int gx = code & 1, gy = (code >> 1) & 1, gz = (code >> 2) & 1;
        double sum = 0.0;
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
                    const long long j = ((long long)zz * g.ny + yy) * g.nx + xx;
                    RTPN_CHECK_PTR(sa + j);
                    RTPN_CHECK_PTR(ss + j);
                    sum += sa[j] + ss[j];
                    ++cnt;
                }
        const double c = sum / cnt;
        for (int h = 0; h < 2; ++h) {
            const double tau = h ? 0.5 * dt : dt;
            F* da = dfac + (long long)(16 * h + 2 * code) * g.V + cell;
            RTPN_CHECK_PTR(da);
            RTPN_CHECK_PTR(da + g.V);
            da[0] = (F)(-tau * exp(-c * tau));
            da[g.V] = (F)(-tau * tau * dE(-c * tau));
        }
    }
    RTPN_CHECK_PTR(sa + cell);
    RTPN_CHECK_PTR(dfac + 33 * g.V + cell);
    const double c0 = sa[cell];
    dfac[(long long)32 * g.V + cell] = (F)(-dt * exp(-c0 * dt));
    dfac[(long long)33 * g.V + cell] = (F)(-dt * dt * dE(-c0 * dt));
}

// The class-cls components grouped by the factors they share: {plane of alpha (FAC_U0 for u_0),
// gacc slot, first, end} per group, then the local indices of every group (host).
struct PullTable {
    std::vector<int> grp, idx;
};
inline PullTable pull_table(const Model& md, int cls) {
    const int a0 = cls == 0 ? 0 : md.ne, na = cls == 0 ? md.ne : md.no;
    std::map<int, std::vector<int>> by_plane;
    for (int t = 0; t < na; ++t) {
        const int a = md.abi_of_internal[a0 + t];
        by_plane[a == 0 ? FAC_U0 : 2 * slot_code(md.comp[a].slot)].push_back(t);
    }
    PullTable p;
    for (const auto& [fp, ts] : by_plane) {
        p.grp.insert(p.grp.end(), {fp, fp == FAC_U0 ? 8 : fp / 2, (int)p.idx.size(), (int)(p.idx.size() + ts.size())});
        p.idx.insert(p.idx.end(), ts.begin(), ts.end());
    }
    return p;
}

// four consecutive floats (16-byte aligned on the device): through the read-only path, plainly
// (memory the same thread rewrites), and a store
RTPN_HD float4 ld4(const float* p) {
    RTPN_CHECK_PTR(p);
    RTPN_CHECK_PTR(p + 3);
#ifdef __CUDA_ARCH__
    return __ldg(reinterpret_cast<const float4*>(p));
#else
    return make_float4(p[0], p[1], p[2], p[3]);
#endif
}
RTPN_HD float4 ld4_rw(const float* p) {
    RTPN_CHECK_PTR(p);
    RTPN_CHECK_PTR(p + 3);
#ifdef __CUDA_ARCH__
    return *reinterpret_cast<const float4*>(p);
#else
    return make_float4(p[0], p[1], p[2], p[3]);
#endif
}
RTPN_HD void st4(float* p, float4 v) {
    RTPN_CHECK_PTR(p);
    RTPN_CHECK_PTR(p + 3);
#ifdef __CUDA_ARCH__
    *reinterpret_cast<float4*>(p) = v;
#else
    p[0] = v.x, p[1] = v.y, p[2] = v.z, p[3] = v.w;
#endif
}
RTPN_HD int ldi(const int* p) {
    RTPN_CHECK_PTR(p);
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// The pull-back through a pass on class A between two stored FP32 states, for the four cells
// c0 .. c0 + 3.  The pass computed u_A' = alpha u_A + beta r_A (Eq. 5), so its residual is
// r_A = (u_A' - alpha u_A) / beta (q included for u_0) and no stencil is needed:
// gacc[slot] += sum_a lam_a (dalpha u_a + dbeta r_a), gq += beta_0 lam_0, w_a = beta_a lam_a.
// lam_a <- alpha_a lam_a is left to the next transposed coupling onto class A.  Where two passes on
// class A follow each other (the odd half passes that close one checkpoint segment and open the
// next), the later one's scaling is still pending: pre_ofs >= 0 gives its factors, lam is scaled
// by them first and stored back.  upre, upost and lam point at class A's first component; w holds
// class A in its local order; grp / idx are a PullTable.  V % 4 == 0.
RTPN_HD void pull_cells(const float* upre, const float* upost, float* lam, float* w, const float* fac,
                        const float* dfac, int fac_ofs, int pre_ofs, const int* grp, int ngroups, const int* idx,
                        long long V, long long c0, double* gacc, double* gq) {
    for (int gi = 0; gi < ngroups; ++gi) {
        const int fp = ldi(grp + 4 * gi), slot = ldi(grp + 4 * gi + 1);
        const int jb = ldi(grp + 4 * gi + 2), je = ldi(grp + 4 * gi + 3);
        const bool u0 = fp == FAC_U0;
        const long long ap = u0 ? FAC_U0 : fp + fac_ofs, dp = u0 ? 32 : fp + fac_ofs;
        float al[4], be[4], da[4], db[4], ib[4], acc[4] = {0.f, 0.f, 0.f, 0.f}, gqa[4] = {0.f, 0.f, 0.f, 0.f};
        float pre[4] = {1.f, 1.f, 1.f, 1.f};
        if (pre_ofs >= 0) {
            const float4 p4 = ld4(fac + (u0 ? (long long)FAC_U0 : (long long)fp + pre_ofs) * V + c0);
            pre[0] = p4.x, pre[1] = p4.y, pre[2] = p4.z, pre[3] = p4.w;
        }
        {
            const float4 a4 = ld4(fac + ap * V + c0), b4 = ld4(fac + (ap + 1) * V + c0);
            const float4 d4 = ld4(dfac + dp * V + c0), e4 = ld4(dfac + (dp + 1) * V + c0);
            al[0] = a4.x, al[1] = a4.y, al[2] = a4.z, al[3] = a4.w;
            be[0] = b4.x, be[1] = b4.y, be[2] = b4.z, be[3] = b4.w;
            da[0] = d4.x, da[1] = d4.y, da[2] = d4.z, da[3] = d4.w;
            db[0] = e4.x, db[1] = e4.y, db[2] = e4.z, db[3] = e4.w;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) ib[c] = 1.f / be[c];
#pragma unroll 2
        for (int j = jb; j < je; ++j) {
            const long long o = (long long)ldi(idx + j) * V + c0;
            const float4 u4 = ld4(upre + o), p4 = ld4(upost + o);
            float4 l4 = ld4_rw(lam + o);
            if (pre_ofs >= 0) {
                l4 = make_float4(pre[0] * l4.x, pre[1] * l4.y, pre[2] * l4.z, pre[3] * l4.w);
                st4(lam + o, l4);
            }
            const float u[4] = {u4.x, u4.y, u4.z, u4.w}, up[4] = {p4.x, p4.y, p4.z, p4.w};
            const float la[4] = {l4.x, l4.y, l4.z, l4.w};
            float wv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float r = fmaf(-al[c], u[c], up[c]) * ib[c];
                acc[c] = fmaf(la[c], fmaf(da[c], u[c], db[c] * r), acc[c]);
                gqa[c] = fmaf(be[c], la[c], gqa[c]);
                wv[c] = be[c] * la[c];
            }
            st4(w + o, make_float4(wv[0], wv[1], wv[2], wv[3]));
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            RTPN_CHECK_PTR(gacc + (long long)slot * V + c0 + c);
            gacc[(long long)slot * V + c0 + c] += (double)acc[c];
            if (u0) {
                RTPN_CHECK_PTR(gq + c0 + c);
                gq[c0 + c] += (double)gqa[c];
            }
        }
    }
}

}  // namespace adj
}  // namespace rtpn
