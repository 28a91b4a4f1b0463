// Register-window substep kernel for a compiled order N (FP32 arithmetic, FP32 or BF16 storage).
//
// One thread owns one cell and advances every component of the target class A by Eq. (5), with the
// dual class B frozen (Eq. 4).  The coupling of Eq. (3) only joins (l, m) to (l +- 1, m) through Mz
// and to (l +- 1, |m| +- 1) through Mx and My, so the sources are swept column by column in |m|:
// every source value is loaded once (plus its one neighbour per axis that a half-grid difference
// needs, Section 2.1), its three differences are formed in registers, and each difference is
// scattered into the accumulators of its <= 10 targets (the unrolled sparse product of Section
// 3.2).  A target column |m| = M is complete once source column M + 1 has been swept, so only three
// columns of accumulators are live: a register window.  Everything indexed by (l, m) is resolved at
// compile time; the coefficients M_d[a][b] * dir come from __constant__ memory and 1/h is applied
// once per target.
//
// Sub-grid slot of (l, M, t): x parity (-1)^M for cos type, -(-1)^M for sin type; y parity +1 for cos,
// -1 for sin; z parity (-1)^(l+M); slot 1 = even parity.  A source on slot 1 along d is read at
// i + e_d by its d-partners (they sit on slot 2), a source on slot 2 at i - e_d.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>
#include <unordered_map>
#include <utility>
#include <vector>

#include "rtpn_internal.h"

namespace rtpn {
namespace win {

// ---------------------------------------------------------------- compile-time structure
__host__ __device__ constexpr int first_l(int M, int P) { return (M % 2 == P) ? M : M + 1; }
__host__ __device__ constexpr int column_len(int N, int M, int P) {
    return first_l(M, P) <= N ? (N - first_l(M, P)) / 2 + 1 : 0;
}
__host__ __device__ constexpr int ntypes(int M) { return M == 0 ? 1 : 2; }
// index of (l, M, t) inside class P in the internal order (M, t, l)
__host__ __device__ constexpr int local_index(int N, int P, int l, int M, int t) {
    int idx = 0;
    for (int m = 0; m < M; ++m) idx += ntypes(m) * column_len(N, m, P);
    return idx + t * column_len(N, M, P) + (l - first_l(M, P)) / 2;
}
__host__ __device__ constexpr int class_size(int N, int P) {
    int n = 0;
    for (int m = 0; m <= N; ++m) n += ntypes(m) * column_len(N, m, P);
    return n;
}
__host__ __device__ constexpr bool valid(int N, int l, int M, int t) {
    return M >= 0 && M <= l && l <= N && (t == 0 || M >= 1) && t >= 0 && t <= 1;
}
__host__ __device__ constexpr int slot_x(int M, int t) { return ((M % 2 == 0) == (t == 0)) ? 1 : 2; }
__host__ __device__ constexpr int slot_y(int t) { return t == 0 ? 1 : 2; }
__host__ __device__ constexpr int slot_z(int l, int M) { return ((l + M) % 2 == 0) ? 1 : 2; }
__host__ __device__ constexpr int slot_code(int l, int M, int t) {
    return (slot_x(M, t) - 1) + 2 * (slot_y(t) - 1) + 4 * (slot_z(l, M) - 1);
}

// Relation k of a source (l, M, t) to one of its <= 10 targets.
//   0,1: z  (l-1, M), (l+1, M)                  same type
//   2,3: x  (l-1, M-1), (l+1, M-1)              same type (M-1 = 0: cos sources only)
//   4,5: x  (l-1, M+1), (l+1, M+1)              same type
//   6,7: y  (l-1, M-1), (l+1, M-1)              other type (M-1 = 0: sin sources only)
//   8,9: y  (l-1, M+1), (l+1, M+1)              other type (M = 0: sin)
struct Target {
    int l, M, t, axis;
    bool ok;
};
__host__ __device__ constexpr Target relation(int N, int l, int M, int t, int k) {
    const int dl = (k % 2 == 0) ? -1 : 1;
    Target r{l + dl, M, t, 2, false};
    if (k <= 1) {
        r = Target{l + dl, M, t, 2, false};
    } else if (k <= 5) {
        const int Mt = k <= 3 ? M - 1 : M + 1;
        r = Target{l + dl, Mt, t, 0, false};
        if (Mt == 0 && t != 0) return r;  // only cos sources reach m = 0 through Mx
    } else {
        const int Mt = k <= 7 ? M - 1 : M + 1;
        int tt = 1 - t;
        if (Mt == 0) {
            if (t != 1) return Target{l + dl, Mt, 0, 1, false};
            tt = 0;
        }
        if (M == 0) tt = 1;
        r = Target{l + dl, Mt, tt, 1, false};
    }
    r.ok = valid(N, r.l, r.M, r.t);
    return r;
}
__host__ __device__ constexpr bool needs_axis(int N, int l, int M, int t, int axis) {
    for (int k = 0; k < 10; ++k) {
        Target r = relation(N, l, M, t, k);
        if (r.ok && r.axis == axis) return true;
    }
    return false;
}

// ---------------------------------------------------------------- compile-time loops
// The per-cell body is __host__ __device__ so that the same code can be run over a grid on the
// host (with bounds-checked memory) when checking it; on the device, loads of the frozen class and
// of the factors go through the read-only path.
#define RTPN_HD __host__ __device__ __forceinline__

template <typename F, int... Is>
RTPN_HD void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int Count, typename F>
RTPN_HD void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, Count>{});
}

#ifndef RTPN_HOST_CHECK
#define RTPN_CHECK_PTR(p) ((void)0)
#endif

RTPN_HD float ro(const float* p) {
    RTPN_CHECK_PTR(p);
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}
template <typename S>
RTPN_HD float load_nc(const S* p);
template <>
RTPN_HD float load_nc<float>(const float* p) { return ro(p); }
template <>
RTPN_HD float load_nc<__nv_bfloat16>(const __nv_bfloat16* p) {
    RTPN_CHECK_PTR(p);
#ifdef __CUDA_ARCH__
    return __bfloat162float(__ldg(p));
#else
    return __bfloat162float(*p);
#endif
}
template <typename S>
RTPN_HD void store(S* p, float v);
template <>
RTPN_HD void store<float>(float* p, float v) {
    RTPN_CHECK_PTR(p);
    *p = v;
}
template <>
RTPN_HD void store<__nv_bfloat16>(__nv_bfloat16* p, float v) {
    RTPN_CHECK_PTR(p);
    *p = __float2bfloat16_rn(v);
}

struct Args {
    void* u;
    const float* fac;
    long long V;
    int nx, ny, nz, bc;
    int fac_ofs;
    float inv_h;        // 1 / h (the constants hold M_d[a][b] * dir without it)
    int tx, ty, tz;     // CTA tile (threads = tx*ty*tz)
    int ntx, nty, ntz;  // tiles per axis
    float sy = 1.f, sz = 1.f;  // h / h_y, h / h_z: the y and z differences' scale (non-cubic cells)
    int aniso = 0;             // factors per (sub-grid, order l): anisotropic scattering
};

// coef[j * 10 + k]: source j (local index in class B), relation k: M_d[a][b] * dir, where dir = +1 if
// the source is read at i + e_d and -1 if at i - e_d; r = -(1/h) * sum coef * (u(neighbour) - u(i)).
// Cell of thread `tid` in block `blk`: tiles are ordered with z fastest, so consecutive blocks are
// z-neighbours and share their planes through L2.
RTPN_HD bool cell_of(const Args& a, int blk, int tid, int* x, int* y, int* z) {
    const int lx = tid % a.tx, ly = (tid / a.tx) % a.ty, lz = tid / (a.tx * a.ty);
    const int bz = blk % a.ntz;
    const int rest = blk / a.ntz;
    const int bx = rest % a.ntx, by = rest / a.ntx;
    *x = bx * a.tx + lx;
    *y = by * a.ty + ly;
    *z = bz * a.tz + lz;
    return *x < a.nx && *y < a.ny && *z < a.nz;
}

// SCALED: non-cubic cells (Section 2.1 divides each difference by its own axis' cell size); the
// y and z differences are scaled by h / h_y and h / h_z, and 1/h (of x) is applied per target.
// ANISO: anisotropic scattering (Section 2, Sigma_tl = Sigma_a + Sigma_s0 - Sigma_sl): every target
// (l, M, t) reads the factors of its own (sub-grid, order l) planes at finish instead of the four
// per-sub-grid pairs (the same factor planes as the generic kernel; u_0 keeps its own).
// Both forms are compiled up to order kExtendedMaxN: P39 runs non-cubic cells on the staged
// kernel, and its window body is the slowest to compile.
constexpr int kExtendedMaxN = 15;
template <int N, int A, typename S, bool SCALED = false, bool ANISO = false>
RTPN_HD void substep_cell(const Args& a, const float* __restrict__ coef, int x, int y, int z) {
    constexpr int B = 1 - A;
    constexpr int NL = N / 2 + 1;
    const long long V = a.V;
    const long long cell = ((long long)z * a.ny + y) * a.nx + x;
    const bool periodic = a.bc == RTPN_BC_PERIODIC;
    // neighbour offsets: [axis][0] = lower (i-1), [axis][1] = upper (i+1)
    int off[3][2];
    bool ok[3][2];
    {
        const int c[3] = {x, y, z};
        const int n[3] = {a.nx, a.ny, a.nz};
        const int stride[3] = {1, a.nx, a.nx * a.ny};
        for (int d = 0; d < 3; ++d) {
            ok[d][0] = c[d] > 0 || periodic;
            off[d][0] = c[d] > 0 ? -stride[d] : (n[d] - 1) * stride[d];
            ok[d][1] = c[d] < n[d] - 1 || periodic;
            off[d][1] = c[d] < n[d] - 1 ? stride[d] : -(n[d] - 1) * stride[d];
        }
    }
    S* u = reinterpret_cast<S*>(a.u);
    const S* srcbase = u + (long long)(B == 0 ? 0 : class_size(N, 0)) * V + cell;
    S* tgtbase = u + (long long)(A == 0 ? 0 : class_size(N, 0)) * V + cell;

    // ---- factors of the four target sub-grids (and u_0)
    float al[8], be[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        al[g] = 0.f;
        be[g] = 0.f;
    }
    // be holds beta / h: the accumulators carry sum coef * (u(neighbour) - u(i)) without 1/h
    static_for<8>([&](auto gi) {
        constexpr int g = decltype(gi)::value;
        constexpr int twos = (g & 1) + ((g >> 1) & 1) + ((g >> 2) & 1);
        if constexpr (twos % 2 == A && !ANISO) {
            al[g] = ro(a.fac + (long long)(a.fac_ofs + 2 * g) * V + cell);
            be[g] = ro(a.fac + (long long)(a.fac_ofs + 2 * g + 1) * V + cell) * a.inv_h;
        }
    });
    float al0 = 0.f, be0 = 0.f, ga0 = 0.f;
    if constexpr (A == 0) {
        al0 = ro(a.fac + (long long)FAC_U0 * V + cell);
        be0 = ro(a.fac + (long long)(FAC_U0 + 1) * V + cell) * a.inv_h;
        ga0 = ro(a.fac + (long long)(FAC_U0 + 2) * V + cell);
    }

    float acc[3][2][NL];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int j = 0; j < NL; ++j) acc[i][t][j] = 0.f;

    // finalize target column M (every contribution is in)
    auto finalize = [&](auto Mi) {
        constexpr int M = decltype(Mi)::value;
        static_for<2>([&](auto ti) {
            constexpr int t = decltype(ti)::value;
            if constexpr (t < ntypes(M)) {
                static_for<NL>([&](auto ji) {
                    constexpr int j = decltype(ji)::value;
                    constexpr int l = first_l(M, A) + 2 * j;
                    if constexpr (l <= N) {
                        constexpr int idx = local_index(N, A, l, M, t);
                        S* p = tgtbase + (long long)idx * V;
                        const float old = load_nc<S>(p);
                        const float r = acc[M % 3][t][j];
                        acc[M % 3][t][j] = 0.f;
                        float nv;
                        if constexpr (A == 0 && l == 0) {
                            nv = fmaf(al0, old, fmaf(-be0, r, ga0));
                        } else if constexpr (ANISO) {
                            constexpr int pl = aniso_plane(N, slot_code(l, M, t), l);
                            const float alv = ro(a.fac + (long long)(a.fac_ofs + pl) * V + cell);
                            const float bev = ro(a.fac + (long long)(a.fac_ofs + pl + 1) * V + cell) * a.inv_h;
                            nv = fmaf(alv, old, -bev * r);
                        } else {
                            constexpr int g = slot_code(l, M, t);
                            nv = fmaf(al[g], old, -be[g] * r);
                        }
                        store<S>(p, nv);
                    }
                });
            }
        });
    };

    static_for<N + 1>([&](auto Mi) {
        constexpr int Ms = decltype(Mi)::value;
        static_for<2>([&](auto ti) {
            constexpr int ts = decltype(ti)::value;
            if constexpr (ts < ntypes(Ms)) {
                static_for<NL>([&](auto ji) {
                    constexpr int js = decltype(ji)::value;
                    constexpr int ls = first_l(Ms, B) + 2 * js;
                    if constexpr (ls <= N) {
                        constexpr int sidx = local_index(N, B, ls, Ms, ts);
                        const S* p = srcbase + (long long)sidx * V;
                        const float c = load_nc<S>(p);
                        float d[3] = {0.f, 0.f, 0.f};
                        constexpr int sl[3] = {slot_x(Ms, ts), slot_y(ts), slot_z(ls, Ms)};
                        static_for<3>([&](auto di) {
                            constexpr int ax = decltype(di)::value;
                            if constexpr (needs_axis(N, ls, Ms, ts, ax)) {
                                constexpr int side = sl[ax] == 1 ? 1 : 0;
                                const float nb = ok[ax][side] ? load_nc<S>(p + off[ax][side]) : 0.f;
                                d[ax] = nb - c;
                                if constexpr (SCALED && ax > 0) d[ax] *= ax == 1 ? a.sy : a.sz;
                            }
                        });
                        static_for<10>([&](auto ki) {
                            constexpr int k = decltype(ki)::value;
                            constexpr Target T = relation(N, ls, Ms, ts, k);
                            if constexpr (T.ok) {
                                constexpr int jt = (T.l - first_l(T.M, A)) / 2;
                                acc[T.M % 3][T.t][jt] =
                                    fmaf(coef[sidx * 10 + k], d[T.axis], acc[T.M % 3][T.t][jt]);
                            }
                        });
                    }
                });
            }
        });
        // target column Ms - 1 has now received every contribution
        if constexpr (Ms >= 1) finalize(std::integral_constant<int, Ms - 1>{});
        if constexpr (Ms == N) finalize(std::integral_constant<int, N>{});
    });
}

// Coefficient table of target class A: for every source j of class 1 - A (internal order) and
// relation k, M_d[a][b] * dir.  Cross-checks the compile-time relations against the model's
// nonzeros; returns false on any mismatch.
inline bool coef_table(const Model& md, int A, std::vector<float>* out) {
    const int N = md.N, B = 1 - A;
    const int base = B == 0 ? 0 : md.ne;
    const int nS = class_size(N, B);
    if (nS != (B == 0 ? md.ne : md.no)) return false;
    std::unordered_map<long long, std::pair<int, double>> nz;
    long long expected = 0;
    for (const auto& e : md.nz) {
        nz[(long long)e.a * md.nc + e.b] = {e.axis, e.v};
        if (md.comp[e.b].cls == B) ++expected;
    }
    out->assign((size_t)nS * 10, 0.f);
    long long found = 0;
    for (int j = 0; j < nS; ++j) {
        const int b = md.abi_of_internal[base + j];
        const Component& c = md.comp[b];
        if (local_index(N, B, c.l, c.M, c.t) != j) return false;
        for (int k = 0; k < 10; ++k) {
            const Target T = relation(N, c.l, c.M, c.t, k);
            if (!T.ok) continue;
            const int a = abi_index(T.l, T.M, T.t);
            auto it = nz.find((long long)a * md.nc + b);
            if (it == nz.end() || it->second.first != T.axis) return false;
            const double dir = c.slot[T.axis] == 1 ? 1.0 : -1.0;
            (*out)[(size_t)j * 10 + k] = (float)(it->second.second * dir);
            ++found;
        }
    }
    return found == expected;
}

}  // namespace win
}  // namespace rtpn
