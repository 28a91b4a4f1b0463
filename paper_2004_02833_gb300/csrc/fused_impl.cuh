// Fused step kernel: the even full step and the odd step after it (Eq. 6 with the odd half steps of
// neighbouring steps merged) in one pass that streams through z.
//
// The odd update at cell i reads the NEW even class at i and at one neighbour per axis (Eq. 4, the
// half-grid differences of Section 2.1), so a CTA that owns a 32 x 8 column of cells computes the
// new even class one plane ahead of its odd update, on its cells plus a one-cell halo in x and y,
// and keeps the last three such planes in a shared-memory ring.  Plane p of the odd class is then
// updated from ring planes p - 1, p, p + 1.  Reads come from the state before the pass and writes go
// to a second buffer, so halo cells recomputed by two CTAs and cells another CTA has already
// updated never race: one read and one write of the state per step instead of two passes that each
// read the whole state and write half of it.
//
// The per-cell arithmetic is that of the register-window kernel (same coefficient tables, same
// column sweep, same order of operations); only where the sources come from differs.  Each phase is
// a __host__ __device__ function of (block, thread) so that a host loop over threads, with the
// barriers between phases, reproduces the kernel when checking it.
#pragma once

#include "window_impl.cuh"

namespace rtpn {
namespace fus {

using win::class_size;
using win::first_l;
using win::load_nc;
using win::local_index;
using win::needs_axis;
using win::ntypes;
using win::relation;
using win::slot_code;
using win::slot_x;
using win::slot_y;
using win::slot_z;
using win::static_for;
using win::store;
using win::Target;

constexpr int TX = 32, TY = 8;           // cells of a CTA in x and y
constexpr int EX = TX + 2, EY = TY + 2;  // the same with the halo of new even values
constexpr int ECELLS = EX * EY;          // ring cells per plane and component
// one thread per haloed cell in the even phase, so that a plane costs one even and one odd cell
// update on every thread's critical path; threads TX * TY and above sit out the odd phase
constexpr int THREADS = (ECELLS + 31) / 32 * 32;

// shared-memory bytes of the ring: three planes of the new even class on the haloed tile
__host__ __device__ constexpr int ring_bytes(int N) { return 3 * class_size(N, 0) * ECELLS * 4; }

struct Args {
    const void* x;     // state before the pass [c][z][y][x], internal order (read only)
    void* y;           // state after the pass (another buffer)
    const float* fac;  // factor planes
    long long V;
    int nx, ny, nz, bc;
    int fac_even;      // factor planes of the even step (full step)
    int fac_odd;       // factor planes of the odd step (full or half step)
    float inv_h;       // 1 / h
    int zc;            // planes per z chunk
    int ntx, nty, nzc; // tiles in x, y; chunks in z
};

struct Tile {
    int x0, y0, z0, z1;
};

// x fastest, then y, then the z chunk: CTAs resident together share halo rows through L2
RTPN_HD Tile tile_of(const Args& a, int blk) {
    Tile t;
    const int bx = blk % a.ntx;
    const int r = blk / a.ntx;
    const int by = r % a.nty;
    const int bz = r / a.nty;
    t.x0 = bx * TX;
    t.y0 = by * TY;
    t.z0 = bz * a.zc;
    t.z1 = t.z0 + a.zc < a.nz ? t.z0 + a.zc : a.nz;
    return t;
}

// ring plane of plane q (q >= z0 - 1)
RTPN_HD int ring_slot(int q, int z0) { return (q - z0 + 1) % 3; }

// host checks of ring indices (no-op in the library)
#ifndef RTPN_CHECK_RING
#define RTPN_CHECK_RING(p) ((void)0)
#endif

RTPN_HD int wrap(int v, int n) {
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// Accumulates, for every target of class A, sum over its sources b of class 1 - A of
// coef * (u_b(neighbour) - u_b(i)), source column |m| by source column, and hands each target to
// fin.apply<l, M, t>(acc) once its last source column has been swept (the register window: only
// three target columns are open at a time).  src.center<j>() and src.nb<j, axis, side>() give the
// source j (local index in class 1 - A) at the cell and at its lower (side 0) or upper (side 1)
// neighbour.
template <int N, int A, typename Src, typename Fin>
RTPN_HD void sweep(const float* __restrict__ coef, const Src& src, const Fin& fin) {
    constexpr int B = 1 - A;
    constexpr int NL = N / 2 + 1;
    float acc[3][2][NL];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int j = 0; j < NL; ++j) acc[i][t][j] = 0.f;

    auto finalize = [&](auto Mi) {
        constexpr int M = decltype(Mi)::value;
        static_for<2>([&](auto ti) {
            constexpr int t = decltype(ti)::value;
            if constexpr (t < ntypes(M)) {
                static_for<NL>([&](auto ji) {
                    constexpr int j = decltype(ji)::value;
                    constexpr int l = first_l(M, A) + 2 * j;
                    if constexpr (l <= N) {
                        fin.template apply<l, M, t>(acc[M % 3][t][j]);
                        acc[M % 3][t][j] = 0.f;
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
                        const float c = src.template center<sidx>();
                        float d[3] = {0.f, 0.f, 0.f};
                        constexpr int sl[3] = {slot_x(Ms, ts), slot_y(ts), slot_z(ls, Ms)};
                        static_for<3>([&](auto di) {
                            constexpr int ax = decltype(di)::value;
                            if constexpr (needs_axis(N, ls, Ms, ts, ax)) {
                                constexpr int side = sl[ax] == 1 ? 1 : 0;
                                d[ax] = src.template nb<sidx, ax, side>() - c;
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
        if constexpr (Ms >= 1) finalize(std::integral_constant<int, Ms - 1>{});
        if constexpr (Ms == N) finalize(std::integral_constant<int, N>{});
    });
}

// ---------------------------------------------------------------- sources
// the odd class of the state before the pass, at a cell of the domain and its neighbours
template <typename S>
struct GlobalSrc {
    const S* base;  // first odd component at the cell
    long long V;
    int off[3][2];
    bool ok[3][2];
    template <int J>
    RTPN_HD float center() const {
        return load_nc<S>(base + (long long)J * V);
    }
    template <int J, int AX, int SIDE>
    RTPN_HD float nb() const {
        return ok[AX][SIDE] ? load_nc<S>(base + (long long)J * V + off[AX][SIDE]) : 0.f;
    }
};

// the new even class in the ring (zeros outside a vacuum domain; wrapped values when periodic)
struct RingSrc {
    const float* lo;   // ring plane p - 1
    const float* mid;  // plane p
    const float* hi;   // plane p + 1
    int e;             // ring cell of the target cell
    template <int J>
    RTPN_HD float center() const {
        RTPN_CHECK_RING(mid + J * ECELLS + e);
        return mid[J * ECELLS + e];
    }
    template <int J, int AX, int SIDE>
    RTPN_HD float nb() const {
        constexpr int step = AX == 0 ? (SIDE ? 1 : -1) : AX == 1 ? (SIDE ? EX : -EX) : 0;
        const float* p = (AX == 2 ? (SIDE ? hi : lo) : mid) + J * ECELLS + e + step;
        RTPN_CHECK_RING(p);
        return *p;
    }
};

// ---------------------------------------------------------------- targets
// Eq. (5) for target (l, M, t) of class A from its old value at the cell (state before the pass):
// new = alpha * old - (beta / h) * acc (+ beta q for u_0).  The value as stored (rounded to S) goes
// to the ring when ring != nullptr and to the output buffer when out != nullptr.
template <int N, int A, typename S>
struct Update {
    const S* old;  // first component of class A at the cell, state before the pass
    S* out;        // first component of class A at the cell, output buffer (or nullptr)
    float* ring;   // ring plane at the ring cell (or nullptr); component stride ECELLS
    long long V;
    float al[8], be[8];
    float al0, be0, ga0;
    template <int l, int M, int t>
    RTPN_HD void apply(float r) const {
        constexpr int idx = local_index(N, A, l, M, t);
        const float o = load_nc<S>(old + (long long)idx * V);
        float nv;
        if constexpr (A == 0 && l == 0) {
            nv = fmaf(al0, o, fmaf(-be0, r, ga0));
        } else {
            constexpr int g = slot_code(l, M, t);
            nv = fmaf(al[g], o, -be[g] * r);
        }
        if (out) store<S>(out + (long long)idx * V, nv);
        if (ring) {
            RTPN_CHECK_RING(ring + idx * ECELLS);
            if constexpr (std::is_same<S, float>::value) {
                ring[idx * ECELLS] = nv;
            } else {
                ring[idx * ECELLS] = __bfloat162float(__float2bfloat16_rn(nv));
            }
        }
    }
};

template <int N, int A, typename S>
RTPN_HD void load_factors(const Args& a, int fac_ofs, long long cell, Update<N, A, S>* u) {
    for (int g = 0; g < 8; ++g) {
        u->al[g] = 0.f;
        u->be[g] = 0.f;
    }
    static_for<8>([&](auto gi) {
        constexpr int g = decltype(gi)::value;
        constexpr int twos = (g & 1) + ((g >> 1) & 1) + ((g >> 2) & 1);
        if constexpr (twos % 2 == A) {
            u->al[g] = win::ro(a.fac + (long long)(fac_ofs + 2 * g) * a.V + cell);
            u->be[g] = win::ro(a.fac + (long long)(fac_ofs + 2 * g + 1) * a.V + cell) * a.inv_h;
        }
    });
    u->al0 = u->be0 = u->ga0 = 0.f;
    if constexpr (A == 0) {
        u->al0 = win::ro(a.fac + (long long)FAC_U0 * a.V + cell);
        u->be0 = win::ro(a.fac + (long long)(FAC_U0 + 1) * a.V + cell) * a.inv_h;
        u->ga0 = win::ro(a.fac + (long long)(FAC_U0 + 2) * a.V + cell);
    }
}

// ---------------------------------------------------------------- phases
// New even class at ring cell e of plane q (unwrapped coordinates x, y, q): into the ring slot, and
// into the output buffer when `own` (a cell of this tile, in the domain, in this CTA's z chunk).
template <int N, typename S>
RTPN_HD void even_cell(const Args& a, const float* __restrict__ coef_e, float* slot, int e, int x, int y,
                       int q, bool own) {
    constexpr int NE = class_size(N, 0);
    const bool periodic = a.bc == RTPN_BC_PERIODIC;
    if (!periodic && (x < 0 || x >= a.nx || y < 0 || y >= a.ny || q < 0 || q >= a.nz)) {
        for (int j = 0; j < NE; ++j) {
            RTPN_CHECK_RING(slot + j * ECELLS + e);
            slot[j * ECELLS + e] = 0.f;
        }
        return;
    }
    const int xw = periodic ? wrap(x, a.nx) : x;
    const int yw = periodic ? wrap(y, a.ny) : y;
    const int zw = periodic ? wrap(q, a.nz) : q;
    const long long V = a.V;
    const long long cell = ((long long)zw * a.ny + yw) * a.nx + xw;
    GlobalSrc<S> src;
    {
        const int c[3] = {xw, yw, zw};
        const int n[3] = {a.nx, a.ny, a.nz};
        const int stride[3] = {1, a.nx, a.nx * a.ny};
        for (int d = 0; d < 3; ++d) {
            src.ok[d][0] = c[d] > 0 || periodic;
            src.off[d][0] = c[d] > 0 ? -stride[d] : (n[d] - 1) * stride[d];
            src.ok[d][1] = c[d] < n[d] - 1 || periodic;
            src.off[d][1] = c[d] < n[d] - 1 ? stride[d] : -(n[d] - 1) * stride[d];
        }
    }
    const S* xs = reinterpret_cast<const S*>(a.x);
    src.base = xs + (long long)NE * V + cell;
    src.V = V;
    Update<N, 0, S> up;
    up.old = xs + cell;
    up.out = own ? reinterpret_cast<S*>(a.y) + cell : nullptr;
    up.ring = slot + e;
    up.V = V;
    load_factors<N, 0, S>(a, a.fac_even, cell, &up);
    sweep<N, 0>(coef_e, src, up);
}

// Even phase of plane q for thread tid: haloed cell tid (row-major over the EX x EY tile).
template <int N, typename S>
RTPN_HD void even_phase(const Args& a, const float* __restrict__ coef_e, float* ring, const Tile& t, int tid,
                        int q) {
    constexpr int NE = class_size(N, 0);
    if (tid >= ECELLS) return;
    float* slot = ring + (long long)ring_slot(q, t.z0) * NE * ECELLS;
    const int ex = tid % EX, ey = tid / EX;
    const int x = t.x0 + ex - 1, y = t.y0 + ey - 1;
    const bool own = q >= t.z0 && q < t.z1 && ex >= 1 && ex <= TX && ey >= 1 && ey <= TY && x < a.nx &&
                     y < a.ny;
    even_cell<N, S>(a, coef_e, slot, tid, x, y, q, own);
}

// Odd phase of plane p (z0 <= p < z1) for thread tid: the odd class at its cell from ring planes
// p - 1, p, p + 1, into the output buffer.
template <int N, typename S>
RTPN_HD void odd_phase(const Args& a, const float* __restrict__ coef_o, const float* ring, const Tile& t,
                       int tid, int p) {
    constexpr int NE = class_size(N, 0);
    if (tid >= TX * TY) return;
    const int lx = tid % TX, ly = tid / TX;
    const int x = t.x0 + lx, y = t.y0 + ly;
    if (x >= a.nx || y >= a.ny) return;
    const long long V = a.V;
    const long long cell = ((long long)p * a.ny + y) * a.nx + x;
    RingSrc src;
    src.lo = ring + (long long)ring_slot(p - 1, t.z0) * NE * ECELLS;
    src.mid = ring + (long long)ring_slot(p, t.z0) * NE * ECELLS;
    src.hi = ring + (long long)ring_slot(p + 1, t.z0) * NE * ECELLS;
    src.e = (ly + 1) * EX + lx + 1;
    Update<N, 1, S> up;
    up.old = reinterpret_cast<const S*>(a.x) + (long long)NE * V + cell;
    up.out = reinterpret_cast<S*>(a.y) + (long long)NE * V + cell;
    up.ring = nullptr;
    up.V = V;
    load_factors<N, 1, S>(a, a.fac_odd, cell, &up);
    sweep<N, 1>(coef_o, src, up);
}

}  // namespace fus
}  // namespace rtpn
