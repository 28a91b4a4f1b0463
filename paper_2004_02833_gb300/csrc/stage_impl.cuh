// TMA-staged substep kernel with a compact column loop (FP32 arithmetic, FP32 or BF16 storage).
//
// Arithmetic as in the register-window kernel (window_impl.cuh): the frozen class is swept column by
// column in |m|; every source value yields three half-grid differences (Section 2.1) that are
// scattered into the accumulators of its <= 10 targets (Eqs. 4-5; Section 3.2's unrolled sparse
// product), and a target column is finished, by Eq. (5), once the next source column is in.  What
// differs:
//
//  * Two threads share a cell, one per target type (cos / sin).  Targets of type T take their z and
//    x differences from sources of type T and their y differences from sources of the other type
//    (Eq. 3's Mx and Mz keep the type, My swaps it), so the split needs no exchange and the two
//    threads carry equal work.  Each thread keeps three columns of N/2 + 1 accumulators.
//  * The column sweep is a runtime loop whose body handles one column for every l slot; the three
//    live target columns are register arrays that shift by one column per iteration, so the body
//    is the same for every column and fits the instruction cache.
//  * A producer warp moves each source column into shared memory with the Tensor Memory Accelerator
//    (cp.async.bulk.tensor): per type and box kind, boxes of E consecutive components of the
//    (type, |m|) run, as many as the column needs.  The TMA unit of an SM spends on the order of
//    60 cycles per box plus a few per box row, so boxes are large (E components) and tiles wide
//    in x (fewer, longer rows); one producer warp issues them.  A column stage holds, per source
//    component, the tile box plus one halo slab on the side its partners read along each axis (x:
//    an aligned 16-byte group, y: one row, z: one plane), and the column's coupling constants (a
//    plain bulk copy).  Periodic halos use wrapped coordinates; vacuum halos use out-of-range
//    coordinates, which the TMA unit fills with zeros.  The same stage carries the tile boxes of
//    the target column it finishes (column i - 1 in stage i; a tile has N + 2 stages).  NB stage
//    buffers form a ring with a full / empty mbarrier pair each, so up to NB - 1 stages are in
//    flight while one is computed.
//
// CTAs are persistent (one per SM) and walk tiles in z-chunked order (z fastest inside a chunk of kz
// tile layers, then x, then y), so the CTAs at work at any time cover a compact block and read one
// another's halos from L2.  Every mbarrier wait is bounded: one that runs out sets a status bit,
// the warp leaves, and the producer waits (bounded) for the copies it issued before the CTA ends.
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

// Enter a compile-time unrolled slot sequence at a runtime slot: `switch (first) {
// RTPN_SLOT_CASES(f) }` runs f(q) for q = first, first + 1, ... 23 (f ignores q past its range), one
// jump per column instead of a test per slot.
#define RTPN_SLOT_CASE(f, q)                   \
    case q:                                    \
        f(std::integral_constant<int, q>{});   \
        [[fallthrough]];
#define RTPN_SLOT_CASES(f)                                                                          \
    RTPN_SLOT_CASE(f, 0) RTPN_SLOT_CASE(f, 1) RTPN_SLOT_CASE(f, 2) RTPN_SLOT_CASE(f, 3)             \
    RTPN_SLOT_CASE(f, 4) RTPN_SLOT_CASE(f, 5) RTPN_SLOT_CASE(f, 6) RTPN_SLOT_CASE(f, 7)             \
    RTPN_SLOT_CASE(f, 8) RTPN_SLOT_CASE(f, 9) RTPN_SLOT_CASE(f, 10) RTPN_SLOT_CASE(f, 11)           \
    RTPN_SLOT_CASE(f, 12) RTPN_SLOT_CASE(f, 13) RTPN_SLOT_CASE(f, 14) RTPN_SLOT_CASE(f, 15)         \
    RTPN_SLOT_CASE(f, 16) RTPN_SLOT_CASE(f, 17) RTPN_SLOT_CASE(f, 18) RTPN_SLOT_CASE(f, 19)         \
    RTPN_SLOT_CASE(f, 20) RTPN_SLOT_CASE(f, 21) RTPN_SLOT_CASE(f, 22) RTPN_SLOT_CASE(f, 23)         \
    default:                                                                                        \
        break;
constexpr int kMaxSlots = 24;
// The same for chunks of kChunk slots: `switch (first / kChunk) { RTPN_CHUNK_CASES(f) }` runs f(c) for
// chunks c = first / kChunk .. 11, so a compiler sees kChunk slots as one straight-line block.
constexpr int kChunk = 2;  // measured: 2 beats 4 and 8 (P39 FP32 45.3 / 46.1 / 47.5 ms per step)
#define RTPN_CHUNK_CASES(f)                                                                        \
    RTPN_SLOT_CASE(f, 0) RTPN_SLOT_CASE(f, 1) RTPN_SLOT_CASE(f, 2) RTPN_SLOT_CASE(f, 3)             \
    RTPN_SLOT_CASE(f, 4) RTPN_SLOT_CASE(f, 5) RTPN_SLOT_CASE(f, 6) RTPN_SLOT_CASE(f, 7)             \
    RTPN_SLOT_CASE(f, 8) RTPN_SLOT_CASE(f, 9) RTPN_SLOT_CASE(f, 10) RTPN_SLOT_CASE(f, 11)           \
    default:                                                                                        \
        break;

constexpr unsigned STATUS_TIMEOUT = 1u;
constexpr unsigned STATUS_CHECK = 2u;  // a self-check failed (builds with RTPN_STAGE_CHECKS)
// coupling constants per source slot, three float4:
//   [0..3] z (l-1), z (l+1), x to column M-1 (l-1), (l+1)     read by the thread of the same type
//   [4..5] x to column M+1 (l-1), (l+1); [6..7] unused        read by the thread of the same type
//   [8..11] y to column M-1 (l-1), (l+1), to M+1 (l-1), (l+1)  read by the thread of the other type
constexpr int CPAD = 12;

// What a pass computes.  FORWARD: targets u_A' = alpha u_A - beta acc (Eq. 5; the u_0 factors for
// l = 0).  ADJ_SOURCES: the transpose of a substep's coupling for the dual multipliers,
// lam_B' = lam_B + acc / h with the sources the weights w_A = beta_A lam_A of the substep on class A
// (same stencil rule and coefficient table as a forward pass on class B: see csrc/adjoint.cu).
// ADJ_TARGETS: the pull-back through a substep on class A of the adjoint's multipliers: from the
// pre-substep state, the forward residual r_A = -acc / h (+ q for u_0), the media gradients
// gacc[slot] += lam_A (dalpha u_A + dbeta r_A) (and gq += beta_0 lam_0), w_A = beta_A lam_A and
// lam_A <- alpha_A lam_A.
constexpr int FORWARD = 0, ADJ_SOURCES = 1, ADJ_TARGETS = 2;

struct Args {
    void* tgt;              // target array (u for a forward pass, lam for ADJ_SOURCES)
    // ADJ_TARGETS only
    float* lam;             // multipliers [nc][V] (internal order), read and scaled in place
    float* wout;            // w of the target class [local index][V]
    const float* dfac;      // dalpha/dc, dbeta/dc planes (same slot layout as the factors; u_0: 32, 33)
    const double* qsrc;     // q per cell (the u_0 source)
    double* gacc;           // [9][V] media-gradient accumulators (slot codes 0..7, u_0)
    double* gq;             // [V] source gradient
    const float* fac;
    const float* coefcol;   // [column 0..N][type][slot q 0..N/2][CPAD] of the source class (0 for l < M)
    const int* colstart;    // [2][N+2]: first local index of column M in class 0 / class 1
    long long V;
    int nx, ny, nz, bc;
    int fac_ofs;
    float inv_h;
    int ntx, nty, ntz;
    int kz;                 // tile layers per z chunk of the walk
    long long tiles;
    const CUtensorMap* maps;  // four tensor maps over the source array: tile, x halo, y halo, z halo
    const CUtensorMap* tmap;  // tile map over the target array
    int src_c0;               // first component of the source class in the source array
    int nc;                   // components (bound of the 4th tensor coordinate)
    unsigned* status;       // device status word (STATUS_TIMEOUT on a wait that ran out)
    unsigned wait_limit;    // try_wait polls (each up to WAIT_HINT_NS) before giving up
    long long skip_stage;   // stage index never issued (a wait that must run out); -1 normally
};

__host__ __device__ constexpr int pad128(int bytes) { return (bytes + 127) / 128 * 128; }

// Components per TMA box along the component axis.  A box lands at a 128-byte aligned shared-memory
// address, so E times the bytes of one component of every box kind (tile, x halo, y halo, z halo)
// must be a multiple of 128; among such E in [emin, 8] the one that holds a run of N/2 + 1 in the
// fewest slots, then in the fewest boxes, is taken (each box costs the TMA unit a fixed overhead,
// so a variant may ask for larger boxes at the price of shared memory).
__host__ __device__ constexpr int box_comps(int N, int tx, int ty, int tz, int es, int emin) {
    const int nl0 = N / 2 + 1;
    const int kinds[4] = {tx * ty * tz * es, (16 / es) * ty * tz * es, tx * tz * es, tx * ty * es};
    int best = 0, best_slots = 1 << 30;
    for (int e = 8; e >= emin; --e) {
        bool ok = true;
        for (int k = 0; k < 4; ++k) ok = ok && (e * kinds[k]) % 128 == 0;
        const int slots = (nl0 + e - 1) / e * e;
        if (ok && slots < best_slots) {
            best = e;
            best_slots = slots;
        }
    }
    return best;  // 0: no aligned box exists for this tile
}
__host__ __device__ constexpr int run_slots(int N, int e) { return e > 0 ? (N / 2 + e) / e * e : 0; }

template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EM = 1>
struct Layout {
    static constexpr int B = 1 - A;
    static constexpr int ES = (int)sizeof(S);
    static constexpr int E = box_comps(N, TX, TY, TZ, ES, EM > N / 2 + 1 ? N / 2 + 1 : EM);  // per box
    static constexpr int NL = run_slots(N, E);              // run slots per type in shared memory
    static constexpr int NG = NL / E;                       // boxes per run, at most
    static constexpr int NLC = N / 2 + 1;                   // coupling-constant slots per type
    static constexpr int HX = 16 / ES;    // x halo: one aligned 16-byte group
    static constexpr int CELLS = TX * TY * TZ;
    static constexpr int CONSUMER_WARPS = 2 * CELLS / 32;
    static constexpr int THREADS = 2 * CELLS + 32;          // two threads per cell + the producer
    // bytes of one component in each box kind
    static constexpr int CTR_BYTES = TX * TY * TZ * ES;
    static constexpr int HX_BYTES = HX * TY * TZ * ES;
    static constexpr int HY_BYTES = TX * TZ * ES;
    static constexpr int HZ_BYTES = TX * TY * ES;
    static constexpr int COMP_BYTES = CTR_BYTES + HX_BYTES + HY_BYTES + HZ_BYTES;
    // regions of one type: the run's tile boxes, then its x, y and z halos
    static constexpr int R_CTR = pad128(NL * CTR_BYTES);
    static constexpr int R_HX = pad128(NL * HX_BYTES);
    static constexpr int R_HY = pad128(NL * HY_BYTES);
    static constexpr int R_HZ = pad128(NL * HZ_BYTES);
    static constexpr int SRC_T = R_CTR + R_HX + R_HY + R_HZ;
    static constexpr int HXO = R_CTR, HYO = R_CTR + R_HX, HZO = R_CTR + R_HX + R_HY;
    static constexpr int COEF_COL = 2 * NLC * CPAD * 4;     // one column's coupling constants
    static constexpr int R_TGT = pad128(NL * CTR_BYTES);     // tile boxes of one type's targets
    // buffer layout: target boxes, type-0 sources, type-1 sources, coupling constants.  A chunked
    // sweep reads up to kChunk - 1 slots (plus one neighbour offset) below a source region; with the
    // targets first, such reads stay on state data (or the zeros the ring starts with) in the same
    // buffer, never on the coupling constants, whose bits need not be finite in the storage type.
    static constexpr int TGTO = 0;
    static constexpr int SRCO = 2 * R_TGT;
    static constexpr int COEFO = SRCO + 2 * SRC_T;
    static constexpr int BUF = COEFO + pad128(COEF_COL);     // one stage buffer
    static constexpr int BARS = pad128(2 * NB * 8);
    static constexpr int BYTES = NB * BUF + BARS + 128;      // ring, mbarriers, base alignment slack
    static_assert(2 * R_TGT >= (kChunk - 1) * CTR_BYTES + TX * TY * ES,
                  "the target region must cover what a chunked sweep reads below the sources");
    static_assert(TX % HX == 0, "tile width must be a multiple of the 16-byte group");
    static_assert(CELLS % 32 == 0, "a type's threads must fill whole warps");
    static_assert(CTR_BYTES % 16 == 0 && HX_BYTES % 16 == 0 && HY_BYTES % 16 == 0 && HZ_BYTES % 16 == 0,
                  "box components must stay 16-byte aligned");
    static_assert(NB >= 2 && NB <= 8, "two to eight stage buffers");
    static_assert(E > 0, "no 128-byte aligned box for this tile");
    static_assert((E * CTR_BYTES) % 128 == 0 && (E * HX_BYTES) % 128 == 0 && (E * HY_BYTES) % 128 == 0 &&
                      (E * HZ_BYTES) % 128 == 0 && BUF % 128 == 0,
                  "every box must land on a 128-byte boundary");
    static constexpr bool FITS = BYTES <= 232448;  // 227 KB of shared memory per CTA
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
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// One poll: the thread may sleep up to WAIT_HINT_NS for the phase to complete (it wakes when it
// does), so a warp that waits for its data spends few issue slots on the poll loop.
constexpr unsigned WAIT_HINT_NS = 2000;
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(WAIT_HINT_NS)
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
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(bar)
        : "memory");
}
// bounded wait on one mbarrier phase; false if it ran out
__device__ __forceinline__ bool wait_phase(unsigned bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i)
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

// Optional self-checks (compile with -DRTPN_STAGE_CHECKS): an index that breaks the layout sets
// STATUS_CHECK and the access is skipped.  status[1] holds the id of the first failed check,
// status[2] a value of it, status[7] the block.
#ifdef RTPN_STAGE_CHECKS
__device__ __forceinline__ bool scheck_fail(unsigned* st, unsigned id, unsigned val, unsigned aux) {
    atomicOr(st, STATUS_CHECK);
    if (atomicCAS(st + 1, 0u, id) == 0u) {
        st[2] = val;
        st[7] = aux;
    }
    return false;
}
#define RTPN_SCHECK_ID(cond, id, val) ((cond) ? true : scheck_fail(a.status, (id), (unsigned)(val), blockIdx.x))
#else
#define RTPN_SCHECK_ID(cond, id, val) true
#endif
#define RTPN_SCHECK(cond) RTPN_SCHECK_ID(cond, __LINE__, 0)

// Tile geometry: origin, valid extents and halo coordinates ([axis][side], side 1 = upper).
struct TileGeo {
    int x0, y0, z0, wx, wy, wz;
    int hc[3][2];
    int hx_start[2], hx_elem[2];
};

// tile t of the walk: chunks of kz z-layers; inside a chunk z fastest, then x, then y
__host__ __device__ __forceinline__ void tile_coords(unsigned t, int ntx, int nty, int ntz, int kzc, int* bx,
                                                     int* by, int* bz) {
    const unsigned per_chunk = (unsigned)kzc * ntx * nty;
    const unsigned full = (unsigned)(ntz / kzc);
    unsigned chunk, r, kz;
    if (t < full * per_chunk) {
        chunk = t / per_chunk;
        r = t - chunk * per_chunk;
        kz = kzc;
    } else {
        chunk = full;
        r = t - full * per_chunk;
        kz = ntz - full * kzc;
    }
    *bz = (int)(chunk * kzc + r % kz);
    const unsigned rest = r / kz;
    *bx = (int)(rest % ntx);
    *by = (int)(rest / ntx);
}

template <int TX, int TY, int TZ, int HX>
__device__ __forceinline__ TileGeo tile_geo(const Args& a, unsigned t) {
    TileGeo g;
    int bx, by, bz;
    tile_coords(t, a.ntx, a.nty, a.ntz, a.kz, &bx, &by, &bz);
    g.x0 = bx * TX;
    g.y0 = by * TY;
    g.z0 = bz * TZ;
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

// The producer warp: issues the copies of every stage of this CTA's sequence into the ring.
template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EM>
__device__ __forceinline__ void stage_producer(const Args& a, unsigned char* bufs, unsigned full0,
                                               unsigned empty0, int total) {
    using L = Layout<N, A, S, TX, TY, TZ, NB, EM>;
    constexpr int B = 1 - A;
    constexpr int NST = N + 2;
    constexpr int E = L::E, NG = L::NG;
    const int lane = threadIdx.x & 31;
    const int cA0 = A == 0 ? 0 : class_size(N, 0);
    const int cB0 = a.src_c0;
    const CUtensorMap* maps = a.maps;
    // first local index of source column i in class B and of target column i - 1 in class A,
    // advanced column by column (no table loads on the producer's path)
    int offB = 0, offA = 0;
    // the maps were written by the host before the launch; make them visible to the async proxy
#pragma unroll
    for (int k = 0; k < 4; ++k)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(maps + k) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(a.tmap) : "memory");

    int s = 0;
    bool failed = false;
    int b = 0, i = 0;
    unsigned ph = 0;  // phase parity of buffer b's current use (flips when b wraps)
    unsigned tile = blockIdx.x;
    TileGeo g = tile_geo<TX, TY, TZ, L::HX>(a, tile);
    for (; s < total; ++s, i = (i == NST - 1) ? 0 : i + 1) {
        if (i == 0 && s > 0) {
            tile += gridDim.x;
            g = tile_geo<TX, TY, TZ, L::HX>(a, tile);
            offB = offA = 0;
        }
        const unsigned full = full0 + 8 * b;
        if (s >= NB) {  // the consumers must have released the buffer's previous stage
            const bool ok = __all_sync(0xffffffffu, wait_phase(empty0 + 8 * b, ph ^ 1u, a.wait_limit));
            if (!ok) {
                failed = true;
                break;
            }
        }
        const int bcur = b;
        if (++b == NB) {
            b = 0;
            ph ^= 1u;
        }
        // the column offsets of stage s; advanced for the next stage before anything can skip ahead
        const int offB_s = offB, offA_s = offA;
        offB += ntypes(i) * column_len(N, i, B);
        if (i >= 1) offA += ntypes(i - 1) * column_len(N, i - 1, A);
        if (s == a.skip_stage) continue;
        unsigned char* buf = bufs + bcur * L::BUF;
        const int len = column_len(N, i, B);     // sources of column i (none at i = N + 1)
        const int nt = len > 0 ? ntypes(i) : 0;  // source types present in the column
        const int nbox = (len + E - 1) / E;
        const int M = i - 1;                     // target column finished in this stage
        const int lenA = M >= 0 ? column_len(N, M, A) : 0;
        const int ntA = lenA > 0 ? ntypes(M) : 0;
        const int nboxA = (lenA + E - 1) / E;
        const unsigned bytes = nt * nbox * E * L::COMP_BYTES + ntA * nboxA * E * L::CTR_BYTES +
                               (nt > 0 ? L::COEF_COL : 0);
        if (lane == 0) mbar_expect_tx(full, bytes);
        __syncwarp();
        // lane j < 8 NG: source box (type j / (4 NG), kind (j / NG) % 4, box j % NG);
        // 8 NG <= j < 10 NG: target box (type (j - 8 NG) / NG, box j % NG)
        for (int j = lane; j < 10 * NG; j += 32) {
            if (j >= 8 * NG) {
                const int t = (j - 8 * NG) / NG, k = j % NG;
                if (t >= ntA || k >= nboxA) continue;
                const int c = cA0 + offA_s + t * lenA + k * E;
                if (!RTPN_SCHECK_ID(c >= 0 && c < a.nc, 111, c)) continue;
                tma_load_4d(smem_addr(buf + L::TGTO + t * L::R_TGT) + k * E * L::CTR_BYTES, a.tmap, g.x0, g.y0,
                            g.z0, c, full);
                continue;
            }
            const int t = j / (4 * NG), kind = (j / NG) % 4, k = j % NG;
            if (t >= nt || k >= nbox) continue;
            const int c = cB0 + offB_s + t * len + k * E;  // first component of the box
            const unsigned d = smem_addr(buf + L::SRCO + t * L::SRC_T);
            if (!RTPN_SCHECK_ID(c >= 0 && c < a.nc, 101, c)) continue;
            if (kind == 0) {
                tma_load_4d(d + k * E * L::CTR_BYTES, maps, g.x0, g.y0, g.z0, c, full);
            } else if (kind == 1) {  // x slot 1 -> partners read i+1 (upper halo)
                const int hxs = dir_x(i, t) > 0 ? g.hx_start[1] : g.hx_start[0];
                tma_load_4d(d + L::HXO + k * E * L::HX_BYTES, maps + 1, hxs, g.y0, g.z0, c, full);
            } else if (kind == 2) {  // cos type reads y+1, sin type y-1
                tma_load_4d(d + L::HYO + k * E * L::HY_BYTES, maps + 2, g.x0, t == 0 ? g.hc[1][1] : g.hc[1][0],
                            g.z0, c, full);
            } else {                 // z slot 1 (l + M even) reads z+1
                tma_load_4d(d + L::HZO + k * E * L::HZ_BYTES, maps + 3, g.x0, g.y0,
                            ((B + i) & 1) == 0 ? g.hc[2][1] : g.hc[2][0], c, full);
            }
        }
        if (lane == 0 && nt > 0)
            bulk_load(smem_addr(buf + L::COEFO), a.coefcol + (long long)i * (2 * L::NLC * CPAD), L::COEF_COL,
                      full);
    }
    if (failed && lane == 0) atomicOr(a.status, STATUS_TIMEOUT);
    // before the CTA ends, the copies of the last stages issued must have landed
    const int first = s > NB ? s - NB : 0;
    for (int r = first; r < s; ++r)
        if (r != a.skip_stage) wait_phase(full0 + 8 * (r % NB), (unsigned)((r / NB) & 1), a.wait_limit);
}

template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EM, int MODE>
__device__ __forceinline__ void stage_kernel_body(const Args& a, unsigned char* smem) {
    using L = Layout<N, A, S, TX, TY, TZ, NB, EM>;
    static_assert(N >= 1, "order N >= 1");
    static_assert((N + 2) / 2 <= kMaxSlots, "slot switch covers N <= 45");
    constexpr int B = 1 - A;
    constexpr int NLA = (N - A) / 2 + 1;   // class-A components of a run, at most
    constexpr int NLB = (N - B) / 2 + 1;   // class-B components of a run, at most
    constexpr int CELLS = L::CELLS;
    constexpr int HX = L::HX;
    constexpr int NST = N + 2;  // stage i: sources of column i (i <= N), targets of column i - 1
    const int cA0 = A == 0 ? 0 : class_size(N, 0);
    const int* colA = a.colstart + A * (N + 2);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const long long V = a.V;

    // TMA writes into shared memory need 128-byte aligned destinations; the dynamic shared memory
    // window is not guaranteed to start on one, so the layout starts at the next 128-byte boundary.
    smem += (128u - (smem_addr(smem) & 127u)) & 127u;
    // zero the ring once: slots a chunked sweep reads below a column's first source
    // (with zero coupling constants) then always hold finite values
    for (int k = tid; k < NB * L::BUF / 16; k += blockDim.x)
        reinterpret_cast<uint4*>(smem)[k] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // before the TMA writes the ring
    unsigned char* bufs = smem;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(bufs + NB * L::BUF);
    const unsigned full0 = smem_addr(&bars[0]), empty0 = smem_addr(&bars[NB]);
    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(full0 + 8 * b, 1);  // the producer's arrive.expect_tx
            mbar_init(empty0 + 8 * b, L::CONSUMER_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int my_tiles = a.tiles > blockIdx.x ? (int)((a.tiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
    const int total = my_tiles * NST;
    if (warp == L::CONSUMER_WARPS) {
        stage_producer<N, A, S, TX, TY, TZ, NB, EM>(a, bufs, full0, empty0, total);
        return;
    }

    // ---- consumers: thread (T, cell) finishes the targets of type T in its cell
    const int T = tid / CELLS, ctid = tid % CELLS;
    const int lx = ctid % TX, ly = (ctid / TX) % TY, lz = ctid / (TX * TY);
    const int my = ((lz * TY + ly) * TX + lx) * L::ES;

    float prev[NLA], cur[NLA], next[NLA];
#pragma unroll
    for (int q = 0; q < NLA; ++q) prev[q] = cur[q] = next[q] = 0.f;

    TileGeo g{};
    bool active = false;
    long long cell = 0;
    float alE = 0.f, beE = 0.f, alO = 0.f, beO = 0.f;  // Eq. (5) factors of columns M even / odd
    float al0 = 0.f, be0 = 0.f, ga0 = 0.f;             // u_0 (class 0, type 0 only)
    // ADJ_TARGETS: factor derivatives, the u_0 source, the multipliers of the target column being
    // finished (prefetched at the top of the stage) and this tile's media-gradient sums
    float daE = 0.f, dbE = 0.f, daO = 0.f, dbO = 0.f, da0 = 0.f, db0 = 0.f, q0s = 0.f;
    float lpre[MODE == ADJ_TARGETS ? NLA : 1];
    float gE = 0.f, gO = 0.f, g0 = 0.f, gqa = 0.f;

    // first local index of target column M in class A, advanced column by column (offA = colstart
    // of the column finished next); component q = 0 of the run (type T, column M) at this cell
    int offA = 0;
    auto tgt_ptr = [&](int M) {
        return reinterpret_cast<S*>(a.tgt) +
               (long long)(cA0 + offA + T * column_len(N, M, A) - first_l(M, A) / 2) * V + cell;
    };

    unsigned tile = blockIdx.x;
    int b = 0;
    unsigned ph = 0;
    for (int s = 0, i = 0; s < total; ++s, i = (i == NST - 1) ? 0 : i + 1) {
        if (i == 0) {  // new tile: geometry, factors
            if (s > 0) tile += gridDim.x;
            g = tile_geo<TX, TY, TZ, HX>(a, tile);
            active = lx < g.wx && ly < g.wy && lz < g.wz;
            cell = ((long long)(g.z0 + lz) * a.ny + (g.y0 + ly)) * a.nx + (g.x0 + lx);
            if (MODE != ADJ_SOURCES && active) {  // the transposed coupling uses no factors
                // sub-grid slot of (l, M, T) in class A: x by (M, T), y by T, z by (A + M)
#pragma unroll
                for (int par = 0; par < 2; ++par) {
                    const int gx = ((par == 0) == (T == 0)) ? 0 : 1;
                    const int gz = ((A + par) & 1) == 0 ? 0 : 1;
                    const int gc = gx + 2 * T + 4 * gz;
                    const float al = __ldg(a.fac + (long long)(a.fac_ofs + 2 * gc) * V + cell);
                    // the forward folds 1/h into beta; the adjoint keeps beta and da, db per slot
                    const float be = __ldg(a.fac + (long long)(a.fac_ofs + 2 * gc + 1) * V + cell) *
                                     (MODE == ADJ_TARGETS ? 1.f : a.inv_h);
                    if (par == 0) {
                        alE = al;
                        beE = be;
                    } else {
                        alO = al;
                        beO = be;
                    }
                    if constexpr (MODE == ADJ_TARGETS) {
                        const float da = __ldg(a.dfac + (long long)(a.fac_ofs + 2 * gc) * V + cell);
                        const float db = __ldg(a.dfac + (long long)(a.fac_ofs + 2 * gc + 1) * V + cell);
                        if (par == 0) {
                            daE = da;
                            dbE = db;
                        } else {
                            daO = da;
                            dbO = db;
                        }
                    }
                }
                if (A == 0 && T == 0) {
                    al0 = __ldg(a.fac + (long long)FAC_U0 * V + cell);
                    be0 = __ldg(a.fac + (long long)(FAC_U0 + 1) * V + cell) * (MODE == ADJ_TARGETS ? 1.f : a.inv_h);
                    ga0 = __ldg(a.fac + (long long)(FAC_U0 + 2) * V + cell);
                    if constexpr (MODE == ADJ_TARGETS) {
                        da0 = __ldg(a.dfac + 32ll * V + cell);
                        db0 = __ldg(a.dfac + 33ll * V + cell);
                        q0s = (float)a.qsrc[cell];
                    }
                }
            }
        }
        const bool fin = active && i >= 1 && (T == 0 || i - 1 >= 1);  // target column i - 1 of type T
        if constexpr (MODE == ADJ_TARGETS) {
            if (fin) {  // the multipliers of column i - 1, for the finish below
                const int M = i - 1, q0 = first_l(M, A) / 2;
                const float* lp = a.lam + (long long)(cA0 + offA + T * column_len(N, M, A) - q0) * V + cell;
#pragma unroll
                for (int q = 0; q < NLA; ++q)
                    if (q >= q0) lpre[q] = __ldg(lp + (long long)q * V);
            }
        }

        if (!__all_sync(0xffffffffu, wait_phase(full0 + 8 * b, ph, a.wait_limit))) {
            if (lane == 0) atomicOr(a.status, STATUS_TIMEOUT);
            break;
        }
        const unsigned char* buf = bufs + b * L::BUF;

        if (active && column_len(N, i, B) > 0) {
            // ---- scatter source column i into prev (i-1), cur (i), next (i+1)
            const int Ms = i;
            const int fq = first_l(Ms, B) / 2;  // run slot of source q is q - fq
            const float* cf = reinterpret_cast<const float*>(buf + L::COEFO);
            static_for<2>([&](auto Ti) {
                constexpr int TT = decltype(Ti)::value;
                if (T != TT) return;
                constexpr int O = 1 - TT;                  // the other type
                const int dz = ((B + Ms) & 1) == 0 ? 1 : -1;
                // a tile one cell thick along an axis always reads that axis' partner from the halo
                const bool inz = TZ > 1 && lz + dz >= 0 && lz + dz < g.wz;
                const int dx = dir_x(Ms, TT);
                const bool inx = lx + dx >= 0 && lx + dx < g.wx;
                constexpr int dy = O == 0 ? 1 : -1;        // the other type's y partner
                const bool iny = TY > 1 && ly + dy >= 0 && ly + dy < g.wy;
                const unsigned char* rb = buf + L::SRCO + TT * L::SRC_T;
                const unsigned char* ro = buf + L::SRCO + O * L::SRC_T;
                // per neighbour: address of run slot -fq (so source q sits at q) and the slot stride
                const unsigned char* pc = rb + my - fq * L::CTR_BYTES;
                const unsigned char* px =
                    inx ? pc + dx * L::ES
                        : rb + L::HXO + ((lz * TY + ly) * HX + (dx > 0 ? g.hx_elem[1] : g.hx_elem[0])) * L::ES -
                              fq * L::HX_BYTES;
                const int sx = inx ? L::CTR_BYTES : L::HX_BYTES;
                const unsigned char* pz =
                    inz ? pc + dz * TX * TY * L::ES : rb + L::HZO + (ly * TX + lx) * L::ES - fq * L::HZ_BYTES;
                const int sz = inz ? L::CTR_BYTES : L::HZ_BYTES;
                const unsigned char* po = ro + my - fq * L::CTR_BYTES;
                const unsigned char* py =
                    iny ? po + dy * TX * L::ES : ro + L::HYO + (lz * TX + lx) * L::ES - fq * L::HY_BYTES;
                const int sy = iny ? L::CTR_BYTES : L::HY_BYTES;
                const float4* cown = reinterpret_cast<const float4*>(cf + TT * L::NLC * CPAD);
                const float4* coth = reinterpret_cast<const float4*>(cf + O * L::NLC * CPAD);
                // sources q = fq .. NLB - 1 (q < fq has l < Ms: not in the column)
                auto sweep = [&](auto own_c, auto oth_c) {
                    constexpr bool OWN = decltype(own_c)::value, OTH = decltype(oth_c)::value;
                    auto slot = [&](auto qi) {
                        constexpr int q = decltype(qi)::value;
                        if constexpr (q < NLB) {
                            constexpr int ls = 2 * q + B;
                            constexpr int lm = (ls - 1) / 2, lp = (ls + 1) / 2;  // acc index of l-1, l+1
                            constexpr bool has_m = ls - 1 >= 0 && lm < NLA;
                            constexpr bool has_p = ls + 1 <= N && lp < NLA;
                            if constexpr (has_m || has_p) {
                                if (!RTPN_SCHECK(q - fq >= -(kChunk - 1) && q - fq < column_len(N, Ms, B))) return;
                                constexpr int am = has_m ? lm : 0, ap = has_p ? lp : 0;
                                if constexpr (OWN) {
                                    const float c = lds<S>(pc, q * L::CTR_BYTES);
                                    const float ddx = lds<S>(px, q * sx) - c;
                                    const float ddz = lds<S>(pz, q * sz) - c;
                                    const float4 k0 = cown[3 * q], k1 = cown[3 * q + 1];
                                    if constexpr (has_m) cur[am] = fmaf(k0.x, ddz, cur[am]);
                                    if constexpr (has_p) cur[ap] = fmaf(k0.y, ddz, cur[ap]);
                                    if constexpr (has_m) prev[am] = fmaf(k0.z, ddx, prev[am]);
                                    if constexpr (has_p) prev[ap] = fmaf(k0.w, ddx, prev[ap]);
                                    if constexpr (has_m) next[am] = fmaf(k1.x, ddx, next[am]);
                                    if constexpr (has_p) next[ap] = fmaf(k1.y, ddx, next[ap]);
                                }
                                if constexpr (OTH) {
                                    const float c = lds<S>(po, q * L::CTR_BYTES);
                                    const float ddy = lds<S>(py, q * sy) - c;
                                    const float4 k2 = coth[3 * q + 2];
                                    if constexpr (has_m) prev[am] = fmaf(k2.x, ddy, prev[am]);
                                    if constexpr (has_p) prev[ap] = fmaf(k2.y, ddy, prev[ap]);
                                    if constexpr (has_m) next[am] = fmaf(k2.z, ddy, next[am]);
                                    if constexpr (has_p) next[ap] = fmaf(k2.w, ddy, next[ap]);
                                }
                            }
                        }
                    };
                    // chunks of kChunk slots from the one holding fq; slots below fq carry zero
                    // coupling constants and read finite (zeroed or earlier) shared memory
                    auto chunk = [&](auto ci) {
                        constexpr int C = decltype(ci)::value;
                        static_for<kChunk>([&](auto ki) {
                            slot(std::integral_constant<int, C * kChunk + decltype(ki)::value>{});
                        });
                    };
                    switch (fq / kChunk) { RTPN_CHUNK_CASES(chunk) }
                };
                // at |m| = 0 only the cos type exists
                if (Ms == 0)
                    sweep(std::integral_constant<bool, TT == 0>{}, std::integral_constant<bool, O == 0>{});
                else
                    sweep(std::true_type{}, std::true_type{});
            });
        }
        if (fin) {
            // ---- finish target column M = i - 1 (its accumulators are in prev), Eq. (5); the old
            // values are the column's tile boxes in this stage
            const int M = i - 1;
            const float alpha = (M & 1) ? alO : alE, beta = (M & 1) ? beO : beE;
            S* tp = tgt_ptr(M);
            (void)RTPN_SCHECK(offA == colA[M]);
            const int q0 = first_l(M, A) / 2;  // targets q = q0 .. NLA - 1 (l >= M)
            const unsigned char* ob = buf + L::TGTO + T * L::R_TGT + my - q0 * L::CTR_BYTES;
            auto tslot = [&](auto qi) {
                constexpr int q = decltype(qi)::value;
                if constexpr (q < NLA) {
                    const float old = lds<S>(ob, q * L::CTR_BYTES);
                    if constexpr (MODE == ADJ_TARGETS) {
                        const float la = lpre[q];
                        const float r = -a.inv_h * prev[q];  // the forward residual (without q)
                        const long long loc = (long long)(offA + T * column_len(N, M, A) - q0 + q) * V + cell;
                        float al, be;
                        if (A == 0 && q == 0 && M == 0) {
                            g0 = fmaf(la, fmaf(da0, old, db0 * (r + q0s)), g0);
                            gqa = fmaf(be0, la, gqa);
                            al = al0;
                            be = be0;
                        } else {
                            const float da = (M & 1) ? daO : daE, db = (M & 1) ? dbO : dbE;
                            const float gv = la * fmaf(da, old, db * r);
                            if (M & 1)
                                gO += gv;
                            else
                                gE += gv;
                            al = alpha;
                            be = beta;
                        }
                        a.wout[loc] = be * la;
                        a.lam[(long long)cA0 * V + loc] = al * la;
                    } else {
                        float nv;
                        if constexpr (MODE == ADJ_SOURCES)
                            nv = fmaf(a.inv_h, prev[q], old);
                        else if (A == 0 && q == 0 && M == 0)
                            nv = fmaf(al0, old, fmaf(-be0, prev[q], ga0));
                        else
                            nv = fmaf(alpha, old, -beta * prev[q]);
                        win::store<S>(tp + (long long)q * V, nv);
                    }
                }
            };
            switch (q0) { RTPN_SLOT_CASES(tslot) }
        }
        // the stage buffer is free once every lane of the warp is past its reads
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * b);
        if (++b == NB) {
            b = 0;
            ph ^= 1u;
        }
        // shift the window: prev <- cur <- next <- 0
#pragma unroll
        for (int q = 0; q < NLA; ++q) {
            prev[q] = cur[q];
            cur[q] = next[q];
            next[q] = 0.f;
        }
        if (i >= 1) offA += ntypes(i - 1) * column_len(N, i - 1, A);
        if constexpr (MODE == ADJ_TARGETS) {
            if (i == NST - 1 && active) {
                // this tile's media-gradient sums: each (cell, slot code) belongs to one thread
#pragma unroll
                for (int par = 0; par < 2; ++par) {
                    const int gx = ((par == 0) == (T == 0)) ? 0 : 1;
                    const int gz = ((A + par) & 1) == 0 ? 0 : 1;
                    a.gacc[(long long)(gx + 2 * T + 4 * gz) * V + cell] += (double)(par == 0 ? gE : gO);
                }
                if (A == 0 && T == 0) {
                    a.gacc[8ll * V + cell] += (double)g0;
                    a.gq[cell] += (double)gqa;
                }
                gE = gO = g0 = gqa = 0.f;
            }
        }
        if (i == NST - 1) {  // tile done: reset the window and the column offset
#pragma unroll
            for (int q = 0; q < NLA; ++q) prev[q] = cur[q] = 0.f;
            offA = 0;
        }
    }
}

}  // namespace stg
}  // namespace rtpn
