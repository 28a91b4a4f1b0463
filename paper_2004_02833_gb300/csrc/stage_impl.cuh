// TMA-staged substep kernel with a compact column loop (FP32 arithmetic, FP32 or BF16 storage).
//
// Arithmetic as in the register-window kernel (window_impl.cuh): one thread per cell of a CTA tile
// sweeps the frozen class column by column in |m| and scatters three half-grid differences per
// source into the accumulators of its <= 10 targets (Eqs. 4-5; Section 3.2's unrolled sparse
// product), a target column being finished once the next source column is in.  Two things differ:
//
//  * The column sweep is a runtime loop whose body handles one column for every (type, l) slot of
//    the class; the three live target columns are three register arrays that shift by one column
//    per iteration.  Slots that do not exist in a column are skipped (sources) or carry zero
//    coefficients (targets), so the body is the same for every column and stays small enough for
//    the instruction cache (the fully unrolled body of the register-window kernel is not).
//  * The data of a column reach shared memory through the Tensor Memory Accelerator
//    (cp.async.bulk.tensor), double buffered: while column M is computed the copies of column M+1
//    are in flight.  A column stage holds, per source component, the tile box plus one halo slab on
//    the side its partners read along each axis (x: an aligned 16-byte group, y: one row, z: one
//    plane), and, per target component of the column being finished, its tile box.  Periodic halos
//    use wrapped coordinates; vacuum halos use out-of-range coordinates, which the TMA unit fills
//    with zeros.  The coupling constants sit in shared memory.
//
// CTAs are persistent (one per SM) and walk tiles in z-fastest order; the stage sequence runs on
// across tiles so the pipeline never drains.  Every mbarrier wait is bounded: one that runs out
// sets a status bit, and the CTA leaves after a second bounded wait for the copies in flight.
#pragma once

#include <cuda.h>

#include "window_impl.cuh"

namespace rtpn {
namespace stg {

using win::class_size;
using win::column_len;
using win::first_l;
using win::ntypes;
using win::static_for;

constexpr unsigned STATUS_TIMEOUT = 1u;
constexpr unsigned STATUS_CHECK = 2u;  // a self-check failed (builds with RTPN_STAGE_CHECKS)
constexpr int CPAD = 12;  // coefficients per source in shared memory (10 used), three float4

struct Args {
    void* u;
    const float* fac;
    const float* coef;      // [class-B source][CPAD] in global memory (copied to shared memory)
    const int* colstart;    // [2][N+2]: first local index of column M in class 0 / class 1
    long long V;
    int nx, ny, nz, bc;
    int fac_ofs;
    float inv_h;
    int ntx, nty, ntz;
    long long tiles;
    const CUtensorMap* maps;  // four tensor maps in global memory: tile, x halo, y halo, z halo
    int nc;                   // components (bound of the 4th tensor coordinate)
    unsigned* status;       // device status word (STATUS_TIMEOUT on a wait that ran out)
    long long wait_limit;   // try_wait polls before giving up
    long long skip_stage;   // global stage index never issued (a wait that must run out); -1 normally
};

__host__ __device__ constexpr int pad128(int bytes) { return (bytes + 127) / 128 * 128; }

template <int N, int A, typename S, int TX, int TY, int TZ>
struct Layout {
    static constexpr int B = 1 - A;
    static constexpr int NL = N / 2 + 1;  // components per (type, |m|) run, at most
    static constexpr int ES = (int)sizeof(S);
    static constexpr int HX = 16 / ES;    // x halo: one aligned 16-byte group
    // bytes of one component in each box kind
    static constexpr int CTR_BYTES = TX * TY * TZ * ES;
    static constexpr int HX_BYTES = HX * TY * TZ * ES;
    static constexpr int HY_BYTES = TX * TZ * ES;
    static constexpr int HZ_BYTES = TX * TY * ES;
    // one TMA box carries NL consecutive components of a run; regions per type t:
    static constexpr int R_CTR = pad128(NL * CTR_BYTES);
    static constexpr int R_HX = pad128(NL * HX_BYTES);
    static constexpr int R_HY = pad128(NL * HY_BYTES);
    static constexpr int R_HZ = pad128(NL * HZ_BYTES);
    static constexpr int SRC_T = R_CTR + R_HX + R_HY + R_HZ;   // source regions of one type
    static constexpr int HXO = R_CTR, HYO = R_CTR + R_HX, HZO = R_CTR + R_HX + R_HY;
    static constexpr int TGT0 = 2 * SRC_T;                       // target regions after the sources
    static constexpr int BUF = TGT0 + 2 * R_CTR;
    static constexpr int SRC_TX = NL * (CTR_BYTES + HX_BYTES + HY_BYTES + HZ_BYTES);  // per run
    static constexpr int TGT_TX = NL * CTR_BYTES;
    static constexpr int COEF = pad128(class_size(N, B) * CPAD * 4);
    static constexpr int BYTES = COEF + 2 * BUF + 128 + 128;  // table, two buffers, mbarriers,
                                                              // and slack to align the base to 128 B
    static_assert(TX % HX == 0, "tile width must be a multiple of the 16-byte group");
    static_assert(CTR_BYTES % 16 == 0 && HX_BYTES % 16 == 0 && HY_BYTES % 16 == 0 && HZ_BYTES % 16 == 0,
                  "box components must stay 16-byte aligned");
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int x, int y, int z,
                                            int c, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(c), "r"(bar)
        : "memory");
}
// bounded wait on one mbarrier phase; false if it ran out
__device__ __forceinline__ bool wait_phase(unsigned bar, unsigned parity, long long limit) {
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <typename S>
__device__ __forceinline__ float lds(const unsigned char* base, int byte_off) {
    if constexpr (sizeof(S) == 4) {
        return *reinterpret_cast<const float*>(base + byte_off);
    } else {
        return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(base + byte_off));
    }
}

// Optional self-checks (compile with -DRTPN_STAGE_CHECKS): an index or alignment that breaks the
// layout sets STATUS_CHECK and the access is skipped.
// With the checks on, status[1..] is a diagnostic record: [1] id of the first failed check,
// [2] a value of it, [3] issue() calls, [4] successful waits, [5] stage of a timeout + 1,
// [6] copies issued.
#ifdef RTPN_STAGE_CHECKS
__device__ __forceinline__ bool scheck_fail(unsigned* st, unsigned id, unsigned val, unsigned aux) {
    atomicOr(st, STATUS_CHECK);
    if (atomicCAS(st + 1, 0u, id) == 0u) {  // the first failure keeps its details
        st[2] = val;
        st[7] = aux;
    }
    return false;
}
#define RTPN_SCHECK_AUX(cond, id, val, aux) ((cond) ? true : scheck_fail(a.status, (id), (unsigned)(val), (unsigned)(aux)))
#define RTPN_SCHECK_ID(cond, id, val) RTPN_SCHECK_AUX(cond, id, val, blockIdx.x)
#define RTPN_SCOUNT(slot) atomicAdd(a.status + (slot), 1u)
#else
#define RTPN_SCHECK_AUX(cond, id, val, aux) true
#define RTPN_SCHECK_ID(cond, id, val) true
#define RTPN_SCOUNT(slot) ((void)0)
#endif
#define RTPN_SCHECK(cond) RTPN_SCHECK_ID(cond, __LINE__, 0)

// Tile geometry: origin, valid extents and halo coordinates ([axis][side], side 1 = upper).
struct TileGeo {
    int x0, y0, z0, wx, wy, wz;
    int hc[3][2];
    int hx_start[2], hx_elem[2];
};

// Tile t (t < 2^31, checked on the host) of the walk: z fastest, then x, then y.  32-bit division:
// this runs once per tile and thread.
template <int TX, int TY, int TZ, int HX>
__device__ __forceinline__ TileGeo tile_geo(const Args& a, unsigned t) {
    TileGeo g;
    const unsigned bz = t % (unsigned)a.ntz;
    const unsigned rest = t / (unsigned)a.ntz;
    g.x0 = (int)(rest % (unsigned)a.ntx) * TX;
    g.y0 = (int)(rest / (unsigned)a.ntx) * TY;
    g.z0 = (int)bz * TZ;
    g.wx = min(TX, a.nx - g.x0);
    g.wy = min(TY, a.ny - g.y0);
    g.wz = min(TZ, a.nz - g.z0);
    const bool periodic = a.bc == RTPN_BC_PERIODIC;
    const int o[3] = {g.x0, g.y0, g.z0}, w[3] = {g.wx, g.wy, g.wz}, n[3] = {a.nx, a.ny, a.nz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int up = o[d] + w[d], lo = o[d] - 1;
        if (periodic) {
            if (up >= n[d]) up -= n[d];
            if (lo < 0) lo += n[d];
        }
        g.hc[d][1] = up;
        g.hc[d][0] = lo;
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int xn = g.hc[0][s];
        const int st = xn >= 0 ? (xn / HX) * HX : -HX;
        g.hx_start[s] = st;
        g.hx_elem[s] = xn - st;
    }
    return g;
}

// Source x slot: 1 (read at i+1 by its partners) iff (M even) == (cos type); z slot: 1 iff l+M even.
__device__ __forceinline__ int dir_x(int M, int t) { return ((M & 1) == 0) == (t == 0) ? 1 : -1; }

// SPLIT threads share a cell: part p owns the targets with l/2 in [p NLP, (p+1) NLP) and sweeps the
// sources that reach them (its range and one neighbouring l on each side), so each thread keeps a
// window of 3 x 2 x NLP accumulators and the CTA runs SPLIT times as many warps on the same tile.
template <int N, int A, typename S, int TX, int TY, int TZ, int SPLIT>
__device__ __forceinline__ void stage_kernel_body(const Args& a, unsigned char* smem) {
    using L = Layout<N, A, S, TX, TY, TZ>;
    constexpr int B = 1 - A;
    constexpr int NL = L::NL;
    constexpr int CELLS = TX * TY * TZ;
    constexpr int NLP = (NL + SPLIT - 1) / SPLIT;
    constexpr int HX = L::HX;
    constexpr int NSTAGE = N + 2;  // stage i: sources of column i (i <= N), targets of column i-1
    const int cA0 = A == 0 ? 0 : class_size(N, 0);
    const int cB0 = B == 0 ? 0 : class_size(N, 0);
    const int* colA = a.colstart + A * (N + 2);
    const int* colB = a.colstart + B * (N + 2);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int part = tid / CELLS, ctid = tid % CELLS;
    const int lx = ctid % TX, ly = (ctid / TX) % TY, lz = ctid / (TX * TY);
    const long long V = a.V;

    // TMA writes into shared memory need 128-byte aligned destinations; the dynamic shared memory
    // window is not guaranteed to start on one, so the layout starts at the next 128-byte boundary.
    smem += (128u - (smem_addr(smem) & 127u)) & 127u;
    float* coef = reinterpret_cast<float*>(smem);
    unsigned char* bufs = smem + L::COEF;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(bufs + 2 * L::BUF);
    const unsigned bar0 = smem_addr(&bars[0]), bar1 = smem_addr(&bars[1]);

    const CUtensorMap* map_ctr = a.maps;
    const CUtensorMap* map_hx = a.maps + 1;
    const CUtensorMap* map_hy = a.maps + 2;
    const CUtensorMap* map_hz = a.maps + 3;

    // coupling constants into shared memory
    for (int i = tid; i < class_size(N, B) * CPAD; i += CELLS * SPLIT) coef[i] = a.coef[i];
    if (tid < 4) {
        // the maps were written by the host before the launch; make them visible to the async proxy
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(a.maps + tid)
                     : "memory");
    }
#ifdef RTPN_STAGE_CHECKS
    if (tid == 0) {
        RTPN_SCHECK_AUX(a.nc == (N + 1) * (N + 1), 121, a.nc, 0);
        RTPN_SCHECK_AUX(colA[0] == 0 && colA[N + 1] == class_size(N, A), 122, colA[N + 1], colA[1]);
        RTPN_SCHECK_AUX(colB[0] == 0 && colB[N + 1] == class_size(N, B), 123, colB[N + 1], colB[1]);
    }
#endif
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // stages of this CTA (the host keeps tiles * NSTAGE below 2^31)
    const int my_tiles = a.tiles > blockIdx.x ? (int)((a.tiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
    const int total = my_tiles * NSTAGE;

    // Issue stage s of this CTA (column stage i of the tile with geometry g): warp 0.  One TMA box
    // per (type, box kind) carries the NL consecutive components of a (type, |m|) run starting at
    // the run's first component: lanes 0-3 the source boxes of type 0, 4-7 of type 1, 8-9 the target
    // boxes of types 0 and 1.
    auto issue = [&](int s, int i, const TileGeo& g) {
        if (s == a.skip_stage) return;
        unsigned char* buf = bufs + (s & 1) * L::BUF;
        const unsigned bar = (s & 1) ? bar1 : bar0;
        const bool src_t[2] = {i <= N && column_len(N, i, B) > 0, i >= 1 && i <= N && column_len(N, i, B) > 0};
        const int M = i - 1;
        const bool tgt_t[2] = {M >= 0 && column_len(N, M, A) > 0, M >= 1 && column_len(N, M, A) > 0};
        const unsigned bytes = (src_t[0] + src_t[1]) * L::SRC_TX + (tgt_t[0] + tgt_t[1]) * L::TGT_TX;
        if (lane == 0) {
            mbar_expect_tx(bar, bytes);
            RTPN_SCOUNT(3);
        }
        __syncwarp();
        if (lane < 8) {
            const int t = lane / 4, kind = lane % 4;
            if (!src_t[t]) return;
            const int c = cB0 + colB[i] + t * column_len(N, i, B);  // first component of the run
            const unsigned d = smem_addr(buf + t * L::SRC_T);
            if (!RTPN_SCHECK_ID(c >= 0 && c < a.nc, 101, c)) return;
            if (!RTPN_SCHECK_ID((d & 127) == 0, 103, d)) return;
            RTPN_SCOUNT(6);
            if (kind == 0) {
                tma_load_4d(d, map_ctr, g.x0, g.y0, g.z0, c, bar);
            } else if (kind == 1) {  // x slot 1 -> partners read i+1 (upper halo)
                const int hxs = dir_x(i, t) > 0 ? g.hx_start[1] : g.hx_start[0];
                if (!RTPN_SCHECK_ID(hxs % HX == 0, 102, hxs)) return;
                tma_load_4d(d + L::HXO, map_hx, hxs, g.y0, g.z0, c, bar);
            } else if (kind == 2) {  // cos type reads y+1, sin type y-1
                tma_load_4d(d + L::HYO, map_hy, g.x0, t == 0 ? g.hc[1][1] : g.hc[1][0], g.z0, c, bar);
            } else {                 // z slot 1 (l + M even) reads z+1
                tma_load_4d(d + L::HZO, map_hz, g.x0, g.y0, ((B + i) & 1) == 0 ? g.hc[2][1] : g.hc[2][0], c,
                            bar);
            }
        } else if (lane < 10) {
            const int t = lane - 8;
            if (!tgt_t[t]) return;
            const int c = cA0 + colA[M] + t * column_len(N, M, A);
            const unsigned d = smem_addr(buf + L::TGT0 + t * L::R_CTR);
            if (!RTPN_SCHECK_ID(c >= 0 && c < a.nc, 111, c)) return;
            if (!RTPN_SCHECK_ID((d & 127) == 0, 113, d)) return;
            RTPN_SCOUNT(6);
            tma_load_4d(d, map_ctr, g.x0, g.y0, g.z0, c, bar);
        }
    };

    float prev[2][NLP], cur[2][NLP], next[2][NLP];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int q = 0; q < NLP; ++q) prev[t][q] = cur[t][q] = next[t][q] = 0.f;

    // geometry of the current tile, computed once per tile (and by warp 0 once more for the first
    // issue into the next tile)
    unsigned cur_tile = blockIdx.x;
    TileGeo g = tile_geo<TX, TY, TZ, HX>(a, cur_tile);
    if (tid < 32 && total > 0) issue(0, 0, g);
    int fail_at = -1;

    bool active = false;
    long long cell = 0;
    float al[8], be[8];
    float al0 = 0.f, be0 = 0.f, ga0 = 0.f;
    int my = 0;
    bool iny[2] = {true, true};

    for (int s = 0, i = 0; s < total; ++s, i = (i == NSTAGE - 1) ? 0 : i + 1) {
        if (i == 0) {  // new tile: geometry, factors, fixed neighbour offsets
            if (s > 0) {
                cur_tile += gridDim.x;
                g = tile_geo<TX, TY, TZ, HX>(a, cur_tile);
            }
            active = lx < g.wx && ly < g.wy && lz < g.wz;
            cell = ((long long)(g.z0 + lz) * a.ny + (g.y0 + ly)) * a.nx + (g.x0 + lx);
            my = ((lz * TY + ly) * TX + lx) * L::ES;
#pragma unroll
            for (int t = 0; t < 2; ++t) {  // y slot is fixed per type: cos reads y+1, sin y-1
                const int dy = t == 0 ? 1 : -1;
                iny[t] = ly + dy >= 0 && ly + dy < g.wy;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) al[k] = be[k] = 0.f;
            if (active) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int twos = (k & 1) + ((k >> 1) & 1) + ((k >> 2) & 1);
                    if (twos % 2 == A) {
                        al[k] = __ldg(a.fac + (long long)(a.fac_ofs + 2 * k) * V + cell);
                        be[k] = __ldg(a.fac + (long long)(a.fac_ofs + 2 * k + 1) * V + cell) * a.inv_h;
                    }
                }
                if (A == 0) {
                    al0 = __ldg(a.fac + (long long)FAC_U0 * V + cell);
                    be0 = __ldg(a.fac + (long long)(FAC_U0 + 1) * V + cell) * a.inv_h;
                    ga0 = __ldg(a.fac + (long long)(FAC_U0 + 2) * V + cell);
                }
            }
        }
        const unsigned bar = (s & 1) ? bar1 : bar0;
        const bool ok = wait_phase(bar, (unsigned)((s >> 1) & 1), a.wait_limit);
        if (__syncthreads_or(!ok)) {
            fail_at = s;
#ifdef RTPN_STAGE_CHECKS
            if (tid == 0) atomicCAS(a.status + 5, 0u, (unsigned)(s + 1));
#endif
            break;
        }
        if (tid == 0) RTPN_SCOUNT(4);
        if (tid < 32 && s + 1 < total) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (i + 1 < NSTAGE) {
                issue(s + 1, i + 1, g);
            } else {
                const TileGeo gn = tile_geo<TX, TY, TZ, HX>(a, cur_tile + gridDim.x);
                issue(s + 1, 0, gn);
            }
        }
        const unsigned char* buf = bufs + (s & 1) * L::BUF;

        if (active && i <= N) {
            // ---- scatter source column i into prev (i-1), cur (i), next (i+1)
            const int Ms = i;
            const int dz = ((B + Ms) & 1) == 0 ? 1 : -1;
            const bool inz = lz + dz >= 0 && lz + dz < g.wz;
            const int fq = first_l(Ms, B) / 2;  // component q' = q - fq inside a run's boxes
            static_for<2>([&](auto ti) {
                constexpr int ts = decltype(ti)::value;
                if (ts == 1 && Ms == 0) return;
                const unsigned char* rb = buf + ts * L::SRC_T;
                const int dx = dir_x(Ms, ts);
                const bool inx = lx + dx >= 0 && lx + dx < g.wx;
                constexpr int dy = ts == 0 ? 1 : -1;
                // per neighbour: address of component q' = 0 and the stride between components
                const unsigned char* pc = rb + my - fq * L::CTR_BYTES;
                const unsigned char* px =
                    inx ? pc + dx * L::ES
                        : rb + L::HXO + ((lz * TY + ly) * HX + (dx > 0 ? g.hx_elem[1] : g.hx_elem[0])) * L::ES -
                              fq * L::HX_BYTES;
                const int sx = inx ? L::CTR_BYTES : L::HX_BYTES;
                const unsigned char* py =
                    iny[ts] ? pc + dy * TX * L::ES : rb + L::HYO + (lz * TX + lx) * L::ES - fq * L::HY_BYTES;
                const int sy = iny[ts] ? L::CTR_BYTES : L::HY_BYTES;
                const unsigned char* pz =
                    inz ? pc + dz * TX * TY * L::ES : rb + L::HZO + (ly * TX + lx) * L::ES - fq * L::HZ_BYTES;
                const int sz = inz ? L::CTR_BYTES : L::HZ_BYTES;
                // local index of slot (ts, q) is cbase + q
                const int cbase = colB[Ms] + ts * column_len(N, Ms, B) - fq;
                static_for<SPLIT>([&](auto pi) {
                constexpr int P = decltype(pi)::value;
                constexpr int QLO = P * NLP, QHI = (P + 1) * NLP < NL ? (P + 1) * NLP : NL;
                if (part != P) return;
                static_for<NL>([&](auto qi) {
                    constexpr int q = decltype(qi)::value;
                    constexpr int ls = 2 * q + B;
                    constexpr int lm = (ls - 1) / 2, lp = (ls + 1) / 2;  // acc index of l-1, l+1
                    constexpr bool has_m = ls - 1 >= 0 && lm >= QLO && lm < QHI;
                    constexpr bool has_p = ls + 1 <= N && lp >= QLO && lp < QHI;
                    if constexpr (ls <= N && (has_m || has_p)) {
                        if (ls < Ms) return;
                        if (!RTPN_SCHECK(q - fq >= 0 && q - fq < NL && cbase + q >= 0 &&
                                         cbase + q < class_size(N, B)))
                            return;
                        const float c = lds<S>(pc, q * L::CTR_BYTES);
                        const float ddx = lds<S>(px, q * sx) - c;
                        const float ddy = lds<S>(py, q * sy) - c;
                        const float ddz = lds<S>(pz, q * sz) - c;
                        const float4* cf = reinterpret_cast<const float4*>(coef + (cbase + q) * CPAD);
                        const float4 k0 = cf[0], k1 = cf[1], k2 = cf[2];
                        constexpr int am = has_m ? lm - QLO : 0, ap = has_p ? lp - QLO : 0;
                        if constexpr (has_m) cur[ts][am] = fmaf(k0.x, ddz, cur[ts][am]);
                        if constexpr (has_p) cur[ts][ap] = fmaf(k0.y, ddz, cur[ts][ap]);
                        if constexpr (has_m) prev[ts][am] = fmaf(k0.z, ddx, prev[ts][am]);
                        if constexpr (has_p) prev[ts][ap] = fmaf(k0.w, ddx, prev[ts][ap]);
                        if constexpr (has_m) next[ts][am] = fmaf(k1.x, ddx, next[ts][am]);
                        if constexpr (has_p) next[ts][ap] = fmaf(k1.y, ddx, next[ts][ap]);
                        if constexpr (has_m) prev[1 - ts][am] = fmaf(k1.z, ddy, prev[1 - ts][am]);
                        if constexpr (has_p) prev[1 - ts][ap] = fmaf(k1.w, ddy, prev[1 - ts][ap]);
                        if constexpr (has_m) next[1 - ts][am] = fmaf(k2.x, ddy, next[1 - ts][am]);
                        if constexpr (has_p) next[1 - ts][ap] = fmaf(k2.y, ddy, next[1 - ts][ap]);
                    }
                });
                });
            });
        }
        if (active && i >= 1) {
            // ---- finish target column i - 1 (its accumulators are in prev)
            const int M = i - 1;
            static_for<2>([&](auto ti) {
                constexpr int t = decltype(ti)::value;
                if (t == 1 && M == 0) return;
                // slot of (l, M, t) for l of class A: x by (M, t), y by t, z by (A + M)
                const int gx = (((M & 1) == 0) == (t == 0)) ? 0 : 1;
                const int gz = ((A + M) & 1) == 0 ? 0 : 1;
                const int gcode = gx + 2 * t + 4 * gz;
                float alpha = 0.f, beta = 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (k == gcode) {
                        alpha = al[k];
                        beta = be[k];
                    }
                S* tptr = reinterpret_cast<S*>(a.u) +
                          (long long)(cA0 + colA[M] + t * column_len(N, M, A) - first_l(M, A) / 2) * V +
                          cell;
                static_for<SPLIT>([&](auto pi) {
                constexpr int P = decltype(pi)::value;
                constexpr int QLO = P * NLP, QHI = (P + 1) * NLP < NL ? (P + 1) * NLP : NL;
                if (part != P) return;
                static_for<NL>([&](auto qi) {
                    constexpr int q = decltype(qi)::value;
                    constexpr int l = 2 * q + A;
                    if constexpr (l <= N && q >= QLO && q < QHI) {
                        if (l < M) return;
                        const long long gi = (long long)(cA0 + colA[M] + t * column_len(N, M, A) -
                                                         first_l(M, A) / 2 + q);
                        if (!RTPN_SCHECK(gi >= cA0 && gi < a.nc && cell >= 0 && cell < V)) return;
                        const float old =
                            lds<S>(buf + L::TGT0 + t * L::R_CTR, my + (q - first_l(M, A) / 2) * L::CTR_BYTES);
                        const float r = prev[t][q - QLO];
                        float nv;
                        if (A == 0 && l == 0 && M == 0)
                            nv = fmaf(al0, old, fmaf(-be0, r, ga0));
                        else
                            nv = fmaf(alpha, old, -beta * r);
                        win::store<S>(tptr + (long long)q * V, nv);
                    }
                });
                });
            });
        }
        // shift the window: prev <- cur <- next <- 0 (also resets a finished tile)
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int q = 0; q < NLP; ++q) {
                prev[t][q] = cur[t][q];
                cur[t][q] = next[t][q];
                next[t][q] = 0.f;
            }
        if (i == NSTAGE - 1) {
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int q = 0; q < NLP; ++q) prev[t][q] = cur[t][q] = 0.f;
        }
        // No barrier here: buffer s & 1 is refilled by the issue of stage s + 2, which warp 0 makes
        // only after the barrier of stage s + 1's wait, when every thread is done with stage s.
    }

    if (fail_at >= 0) {
        if (tid == 0) atomicOr(a.status, STATUS_TIMEOUT);
        // Only the copies of the stage that timed out can still be in flight (the next stage is
        // issued after a successful wait); give them one more bounded wait before leaving.
        wait_phase((fail_at & 1) ? bar1 : bar0, (unsigned)((fail_at >> 1) & 1), a.wait_limit);
        __syncthreads();
    }
}

}  // namespace stg
}  // namespace rtpn
