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
//  * A producer warp moves each column into shared memory with the Tensor Memory Accelerator
//    (cp.async.bulk.tensor): one box per (type, box kind) holding all E components of the
//    (type, |m|) run at once (a tensor map per box length E), so a column stage costs about fifteen
//    TMA operations.  Every box kind has the same volume per component, U = TY * TX elements:
//    the tile as TZ plane boxes [E][1][TY][TX], the y halo row [E][TZ][1][TX], the z halo plane
//    [E][1][TY][TX] and the x halo [E][TZ][RY][XW] (XW * RY = TX: an aligned group of XW columns
//    around the neighbour the partners read, with RY >= TY rows).  So component q of every region
//    sits at q * U elements and each thread reaches all its operands through a few base addresses
//    fixed once per column plus compile-time offsets: no address arithmetic per slot.  Periodic
//    halos use wrapped coordinates; vacuum halos use out-of-range coordinates, which the TMA unit
//    fills with zeros.  The same stage carries the tile boxes of the target column it finishes
//    (column i - 1 in stage i; a tile has N + 2 stages) and the column's coupling constants (a
//    plain bulk copy).  NB stage buffers form a ring with a full / empty mbarrier pair each, so up
//    to NB - 1 stages are in flight while one is computed.
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
constexpr int kChunk = 2;
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
// lam_B' = alpha_B lam_B + acc / h with the sources the weights w_A = beta_A lam_A of the substep on
// class A (same stencil rule and coefficient table as a forward pass on class B: see
// csrc/adjoint.cu); alpha_B, when factors are given, is the factor of the later substep on class B
// whose pull-back lam_B <- alpha_B lam_B is folded in here.
constexpr int FORWARD = 0, ADJ_SOURCES = 1;

// Tensor maps of one array: kind k in {MAP_PLANE, MAP_YROW, MAP_XGRP} for every box length
// E = EQ, 2 EQ, ..., NL (index k * nmaps + E / EQ - 1).
constexpr int MAP_PLANE = 0;  // [E][1][TY][TX]: a tile plane or the z halo plane (also target boxes)
constexpr int MAP_YROW = 1;   // [E][TZ][1][TX]: the y halo row
constexpr int MAP_XGRP = 2;   // [E][TZ][RY][XW]: the x halo group
constexpr int MAP_KINDS = 3;

struct Args {
    void* tgt;              // target array written (u for a forward pass, lam for ADJ_SOURCES)
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
    const CUtensorMap* maps;  // MAP_KINDS * nmaps tensor maps over the source array
    const CUtensorMap* tmap;  // nmaps MAP_PLANE maps over the target array
    int src_c0;               // first component of the source class in the source array
    int nc;                   // components (bound of the 4th tensor coordinate)
    unsigned* status;       // device status word (STATUS_TIMEOUT on a wait that ran out)
    unsigned wait_limit;    // try_wait polls (each up to WAIT_HINT_NS) before giving up
    long long skip_stage;   // stage index never issued (a wait that must run out); -1 normally
};

__host__ __device__ constexpr int pad128(int bytes) { return (bytes + 127) / 128 * 128; }

// Width XW of the x halo box: the widest group of 16-byte aligned columns that divides TX and
// leaves RY = TX / XW >= TY rows (so the box volume per component is TZ * TX = U when TY == TZ).
__host__ __device__ constexpr int xhalo_width(int tx, int ty, int es) {
    int best = 0;
    for (int w = 16 / es; w <= tx; w += 16 / es)
        if (tx % w == 0 && tx / w >= ty) best = w;
    return best;
}
// slots of a run in shared memory: the longest run N/2 + 1 rounded up to a multiple of eq
__host__ __device__ constexpr int run_slots(int N, int eq) { return (N / 2 + 1 + eq - 1) / eq * eq; }

template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EQ = 1>
struct Layout {
    static constexpr int B = 1 - A;
    static constexpr int ES = (int)sizeof(S);
    static constexpr int G = 16 / ES;                 // elements of an aligned 16-byte group
    static constexpr int NL = run_slots(N, EQ);       // run slots per region
    static constexpr int NMAP = NL / EQ;              // box lengths (tensor maps) per kind
    static constexpr int NLC = N / 2 + 1;             // coupling-constant slots per type
    static constexpr int U = TY * TX;                 // elements of one component in every box
    static constexpr int UB = U * ES;
    static constexpr int XW = xhalo_width(TX, TY, ES);
    static constexpr int RY = XW > 0 ? TX / XW : 1;
    static constexpr int CELLS = TX * TY * TZ;
    static constexpr int CONSUMER_WARPS = 2 * CELLS / 32;
    static constexpr int THREADS = 2 * CELLS + 32;   // two threads per cell + the producer
    static constexpr int REG = pad128(NL * UB);       // one region: NL components of one box kind
    // regions of one type's sources: TZ tile planes, then the y halo, z halo and x halo
    static constexpr int KY = TZ, KZ = TZ + 1, KX = TZ + 2, NKIND = TZ + 3;
    static constexpr int SRC_T = NKIND * REG;
    static constexpr int TGT_T = TZ * REG;            // tile planes of one type's targets
    static constexpr int COEF_COL = 2 * NLC * CPAD * 4;  // one column's coupling constants
    // buffer layout: target planes, type-0 sources, type-1 sources, coupling constants.  A chunked
    // sweep reads up to kChunk - 1 slots below a source region; with the targets first, such reads
    // stay on state data (or the zeros the ring starts with) in the same buffer, never on the
    // coupling constants, whose bits need not be finite in the storage type.
    static constexpr int TGTO = 0;
    static constexpr int SRCO = 2 * TGT_T;
    static constexpr int COEFO = SRCO + 2 * SRC_T;
    static constexpr int BUF = COEFO + pad128(COEF_COL);  // one stage buffer
    static constexpr int BARS = pad128(2 * NB * 8);
    static constexpr int BYTES = NB * BUF + BARS + 128;   // ring, mbarriers, base alignment slack
    static_assert(TY == TZ, "every box kind has the volume TY * TX per component only if TY == TZ");
    static_assert(TX % G == 0, "tile width must be a multiple of the 16-byte group");
    static_assert(CELLS % 32 == 0, "a type's threads must fill whole warps");
    static_assert(NB >= 2 && NB <= 8, "two to eight stage buffers");
    static_assert(REG >= (kChunk - 1) * UB, "a region must cover what a chunked sweep reads below the next");
    // the ring fits 227 KB of shared memory per CTA, and an x halo group exists for this element
    // size (a tile too narrow for RY >= TY rows of 16-byte groups is compiled for FP32 only)
    static constexpr bool FITS = BYTES <= 232448 && XW > 0;
};

// The coupling constants of the staged kernel (host; the library and its host check program):
// per target class A, the constants of the source class by column, type and slot q
// ([N+1][2][N/2+1][CPAD], layout above; slots of l < M stay zero, so a sweep may start at a slot
// boundary below the column), from the model's coupling (win::coef_table).  The kernel applies
// 1/h of x; the y and z constants carry sy = h / h_y and sz = h / h_z (exactly 1 for cubic
// cells).  col: the first local index of column M in class P at col[P (N + 2) + M].
inline bool coupling_tables(const Model& md, double sy, double sz, std::vector<float> tab[2], std::vector<int>* col) {
    const int N = md.N, nl = N / 2 + 1;
    col->assign(2 * (N + 2), 0);
    for (int P = 0; P < 2; ++P) {
        int acc = 0;
        for (int M = 0; M <= N + 1; ++M) {
            (*col)[P * (N + 2) + M] = acc;
            if (M <= N) acc += ntypes(M) * column_len(N, M, P);
        }
    }
    for (int A = 0; A < 2; ++A) {
        const int B = 1 - A;
        std::vector<float> t10;  // [local source index of class B][10]
        if (!win::coef_table(md, A, &t10)) return false;
        tab[A].assign((size_t)(N + 1) * 2 * nl * CPAD, 0.f);
        for (int M = 0; M <= N; ++M)
            for (int t = 0; t < ntypes(M); ++t)
                for (int j = 0; j < column_len(N, M, B); ++j) {
                    const int src = (*col)[B * (N + 2) + M] + t * column_len(N, M, B) + j;
                    const int q = first_l(M, B) / 2 + j;  // the source's slot (l - B) / 2
                    float* d = &tab[A][(((size_t)M * 2 + t) * nl + q) * CPAD];
                    const float* kk = &t10[(size_t)src * 10];
                    for (int r = 0; r < 2; ++r) d[r] = (float)(kk[r] * sz);          // z
                    for (int r = 2; r < 6; ++r) d[r] = kk[r];                        // x to M-1, M+1
                    for (int r = 0; r < 4; ++r) d[8 + r] = (float)(kk[6 + r] * sy);  // y to M-1, M+1
                }
    }
    return true;
}

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

// a stored value at base + byte_off of a stage buffer, as FP32 (host and device: the host check
// program runs the consumers' column work over a bounds-checked copy of the buffer)
template <typename S>
RTPN_HD float lds(const unsigned char* base, int byte_off) {
    RTPN_CHECK_PTR(base + byte_off);
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

// Tile geometry: origin, valid extents, halo coordinates ([axis][side], side 1 = upper) and, per
// side, the origin of the x halo group box and the element of the neighbour column inside it.
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

// G: elements of a 16-byte group (the x halo box starts on one)
template <int TX, int TY, int TZ, int G>
__host__ __device__ __forceinline__ TileGeo tile_geo(const Args& a, unsigned t) {
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
    // the neighbour column xn sits at element xn - start of a box that starts on the group holding it
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int xn = g.hc[0][s];
        const int st = xn >= 0 ? (xn / G) * G : -G;
        g.hx_start[s] = st;
        g.hx_elem[s] = xn - st;
    }
    return g;
}

// Source x slot: 1 (read at i+1 by its partners) iff (M even) == (cos type); z slot: 1 iff l+M even.
__host__ __device__ __forceinline__ int dir_x(int M, int t) { return ((M & 1) == 0) == (t == 0) ? 1 : -1; }

// ---------------------------------------------------------------- the stage plan
// One TMA box of a stage: which tensor map (array, kind, box length), its start coordinates and
// where it lands in the stage buffer.  Host and device: the producer issues it, the host check
// program copies it.
struct BoxJob {
    int valid;    // 0: this job issues nothing in this stage
    int target;   // 1: a plane box of the target array (map a.tmap + emap), 0: of the source array
    int kind;     // MAP_PLANE, MAP_YROW or MAP_XGRP (source array)
    int emap;     // box length index: E = EQ * (emap + 1) components
    int x, y, z, c;
    int dst;      // byte offset of the box in the stage buffer
};

// The runs of stage i, the same for every box of the stage: source column i of class B (length,
// types present) and target column i - 1 of class A.
struct StageRuns {
    int len, nt, lenA, ntA;
};
template <int N, int A>
RTPN_HD StageRuns stage_runs(int i) {
    constexpr int B = 1 - A;
    StageRuns r;
    r.len = column_len(N, i, B);          // none at i = N + 1
    r.nt = r.len > 0 ? ntypes(i) : 0;
    r.lenA = i >= 1 ? column_len(N, i - 1, A) : 0;
    r.ntA = r.lenA > 0 ? ntypes(i - 1) : 0;
    return r;
}

// Box j of stage i (runs r) of the tile with geometry g; offB_s and offA_s are the first local
// indices of source column i in class B and of target column i - 1 in class A.  Jobs
// 0 .. 2 NKIND - 1: source boxes (type j / NKIND, kind j % NKIND: TZ tile planes, the y halo row,
// the z halo plane, the x halo group); then the target planes (type, plane).
template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EQ>
RTPN_HD BoxJob stage_box(const Args& a, const TileGeo& g, int i, const StageRuns& r, int offA_s, int offB_s, int j) {
    using L = Layout<N, A, S, TX, TY, TZ, NB, EQ>;
    constexpr int B = 1 - A;
    constexpr int NK = L::NKIND;
    BoxJob bj{0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (j >= 2 * NK) {  // target plane lz of type t
        const int t = (j - 2 * NK) / TZ, lz = (j - 2 * NK) % TZ;
        if (j >= 2 * NK + 2 * TZ || t >= r.ntA) return bj;
        bj.valid = 1;
        bj.target = 1;
        bj.kind = MAP_PLANE;
        bj.emap = (r.lenA + EQ - 1) / EQ - 1;
        bj.x = g.x0;
        bj.y = g.y0;
        bj.z = g.z0 + lz;
        bj.c = (A == 0 ? 0 : class_size(N, 0)) + offA_s + t * r.lenA;
        bj.dst = L::TGTO + t * L::TGT_T + lz * L::REG;
        return bj;
    }
    const int t = j / NK, k = j % NK;
    if (t >= r.nt) return bj;
    bj.valid = 1;
    bj.emap = (r.len + EQ - 1) / EQ - 1;
    bj.c = a.src_c0 + offB_s + t * r.len;  // first component of the run
    bj.dst = L::SRCO + t * L::SRC_T + k * L::REG;
    bj.x = g.x0;
    bj.y = g.y0;
    bj.z = g.z0;
    if (k < TZ) {               // tile plane z0 + k
        bj.kind = MAP_PLANE;
        bj.z = g.z0 + k;
    } else if (k == L::KY) {    // cos-type sources are read at y+1, sin-type at y-1
        bj.kind = MAP_YROW;
        bj.y = t == 0 ? g.hc[1][1] : g.hc[1][0];
    } else if (k == L::KZ) {    // z slot 1 (l + M even) is read at z+1
        bj.kind = MAP_PLANE;
        bj.z = ((B + i) & 1) == 0 ? g.hc[2][1] : g.hc[2][0];
    } else {                    // x slot 1 is read at x+1 (upper halo group)
        bj.kind = MAP_XGRP;
        bj.x = dir_x(i, t) > 0 ? g.hx_start[1] : g.hx_start[0];
    }
    return bj;
}

// bytes the boxes and the coupling constants of a stage with runs r bring into the buffer
template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EQ>
RTPN_HD unsigned stage_bytes(const StageRuns& r) {
    using L = Layout<N, A, S, TX, TY, TZ, NB, EQ>;
    const int ebox = (r.len + EQ - 1) / EQ * EQ, eboxA = (r.lenA + EQ - 1) / EQ * EQ;
    return (unsigned)((r.nt * L::NKIND * ebox + r.ntA * TZ * eboxA) * L::UB) + (r.nt > 0 ? (unsigned)L::COEF_COL : 0u);
}

// The producer warp: issues the copies of every stage of this CTA's sequence into the ring.
template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EQ>
__device__ __forceinline__ void stage_producer(const Args& a, unsigned char* bufs, unsigned full0,
                                               unsigned empty0, int total) {
    using L = Layout<N, A, S, TX, TY, TZ, NB, EQ>;
    constexpr int B = 1 - A;
    constexpr int NST = N + 2;
    constexpr int NJOB = 2 * L::NKIND + 2 * TZ;  // source boxes (type, kind), then target planes (type, z)
    static_assert(NJOB <= 32, "one box per lane");
    const int lane = threadIdx.x & 31;
    const CUtensorMap* maps = a.maps;
    // first local index of source column i in class B and of target column i - 1 in class A,
    // advanced column by column (no table loads on the producer's path)
    int offB = 0, offA = 0;
    // the maps were written by the host before the launch; make them visible to the async proxy
    for (int k = 0; k < MAP_KINDS * L::NMAP; ++k)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(maps + k) : "memory");
    for (int k = 0; k < L::NMAP; ++k)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(a.tmap + k) : "memory");

    int s = 0;
    bool failed = false;
    int b = 0, i = 0;
    unsigned ph = 0;  // phase parity of buffer b's current use (flips when b wraps)
    unsigned tile = blockIdx.x;
    TileGeo g = tile_geo<TX, TY, TZ, L::G>(a, tile);
    for (; s < total; ++s, i = (i == NST - 1) ? 0 : i + 1) {
        if (i == 0 && s > 0) {
            tile += gridDim.x;
            g = tile_geo<TX, TY, TZ, L::G>(a, tile);
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
        // one lane issues the stage: the box list is unrolled at compile time, so the kind of every
        // box and its tensor map are fixed per box and all operands are the same for the warp
        if (lane == 0) {
            const StageRuns runs = stage_runs<N, A>(i);
            mbar_expect_tx(full, stage_bytes<N, A, S, TX, TY, TZ, NB, EQ>(runs));
            static_for<NJOB>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                const BoxJob bj = stage_box<N, A, S, TX, TY, TZ, NB, EQ>(a, g, i, runs, offA_s, offB_s, j);
                // sources: components of the source array (a.nc); targets: of a full state array (u or lam)
                const int cmax = bj.target ? class_size(N, 0) + class_size(N, 1) : a.nc;
                if (bj.valid && RTPN_SCHECK_ID(bj.c >= 0 && bj.c < cmax && (bj.emap + 1) * EQ <= L::NL, 101, bj.c)) {
                    const CUtensorMap* mp = bj.target ? a.tmap + bj.emap : maps + bj.kind * L::NMAP + bj.emap;
                    tma_load_4d(smem_addr(buf + bj.dst), mp, bj.x, bj.y, bj.z, bj.c, full);
                }
            });
            if (runs.nt > 0)
                bulk_load(smem_addr(buf + L::COEFO), a.coefcol + (long long)i * (2 * L::NLC * CPAD), L::COEF_COL,
                          full);
        }
        __syncwarp();
    }
    if (failed && lane == 0) atomicOr(a.status, STATUS_TIMEOUT);
    // before the CTA ends, the copies of the last stages issued must have landed
    const int first = s > NB ? s - NB : 0;
    for (int r = first; r < s; ++r)
        if (r != a.skip_stage) wait_phase(full0 + 8 * (r % NB), (unsigned)((r / NB) & 1), a.wait_limit);
}

// ---------------------------------------------------------------- the consumers' column work
// Byte offsets in a stage buffer of a consumer thread's operands, fixed per tile: its own-type
// source, the other type's source and its y partner, and per parity p of the source column the
// x and z partners.  Thread (T, cell (lx, ly, lz)) finishes the targets of type T of its cell.
struct Operands {
    int c, o, y, x0, x1, z0, z1;
};

template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EQ>
RTPN_HD Operands operand_offsets(const TileGeo& g, int T, int lx, int ly, int lz) {
    using L = Layout<N, A, S, TX, TY, TZ, NB, EQ>;
    constexpr int B = 1 - A, ES = L::ES, REG = L::REG;
    const int cp = (ly * TX + lx) * ES;             // the cell in a tile plane region (per component)
    const int rbo = L::SRCO + T * L::SRC_T;         // own-type sources (z and x partners)
    const int roo = L::SRCO + (1 - T) * L::SRC_T;   // other-type sources (y partners)
    const int dy = T == 0 ? -1 : 1;                 // cos-type sources are read at y+1, sin-type at y-1
    Operands op;
    op.c = rbo + lz * REG + cp;
    op.o = roo + lz * REG + cp;
    op.y = (ly + dy >= 0 && ly + dy < g.wy) ? op.o + dy * TX * ES : roo + L::KY * REG + (lz * TX + lx) * ES;
    int xo[2], zo[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int dx = dir_x(p, T);
        xo[p] = (lx + dx >= 0 && lx + dx < g.wx)
                    ? op.c + dx * ES
                    : rbo + L::KX * REG + ((lz * L::RY + ly) * L::XW + (dx > 0 ? g.hx_elem[1] : g.hx_elem[0])) * ES;
        const int dz = ((B + p) & 1) == 0 ? 1 : -1;
        zo[p] = (lz + dz >= 0 && lz + dz < g.wz) ? op.c + dz * REG : rbo + L::KZ * REG + cp;
    }
    op.x0 = xo[0];
    op.x1 = xo[1];
    op.z0 = zo[0];
    op.z1 = zo[1];
    return op;
}

// Scatter source column i of a stage buffer into the accumulators of target columns i - 1 (prev),
// i (cur) and i + 1 (next) of type T: every source value yields its half-grid differences
// (Section 2.1), each scattered into its <= 10 targets with the column's coupling constants
// (Eqs. 4-5).  At |m| = 0 only the cos type exists: the absent type's constants are zero (its
// regions hold earlier, finite data), so the same sweep serves every column.  Sources
// q = fq .. N/2 (q < fq has l < i: not in the column) are entered at the chunk of kChunk slots
// holding fq; slots below fq carry zero constants and read finite shared memory.
template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EQ>
RTPN_HD void sweep_column(const unsigned char* buf, const Operands& op, int T, int i,
                          float (&prev)[(N - A) / 2 + 1], float (&cur)[(N - A) / 2 + 1],
                          float (&next)[(N - A) / 2 + 1]) {
    using L = Layout<N, A, S, TX, TY, TZ, NB, EQ>;
    constexpr int B = 1 - A, UB = L::UB;
    constexpr int NLA = (N - A) / 2 + 1, NLB = (N - B) / 2 + 1;
    const int fq = first_l(i, B) / 2;  // run slot of source q is q - fq
    const int sh = -fq * UB;           // so source q sits at q * UB from each base
    const unsigned char* pc = buf + op.c + sh;
    const unsigned char* px = buf + ((i & 1) ? op.x1 : op.x0) + sh;
    const unsigned char* pz = buf + ((i & 1) ? op.z1 : op.z0) + sh;
    const unsigned char* po = buf + op.o + sh;
    const unsigned char* py = buf + op.y + sh;
    const float* cf = reinterpret_cast<const float*>(buf + L::COEFO);
    const float4* kown = reinterpret_cast<const float4*>(cf + T * L::NLC * CPAD);
    const float4* koth = reinterpret_cast<const float4*>(cf + (1 - T) * L::NLC * CPAD);
    auto slot = [&](auto qi) {
        constexpr int q = decltype(qi)::value;
        if constexpr (q < NLB) {
            constexpr int ls = 2 * q + B;
            constexpr int lm = (ls - 1) / 2, lp = (ls + 1) / 2;  // acc index of l-1, l+1
            constexpr bool has_m = ls - 1 >= 0 && lm < NLA;
            constexpr bool has_p = ls + 1 <= N && lp < NLA;
            if constexpr (has_m || has_p) {
                constexpr int am = has_m ? lm : 0, ap = has_p ? lp : 0;
                const float c = lds<S>(pc, q * UB);
                const float ddx = lds<S>(px, q * UB) - c;
                const float ddz = lds<S>(pz, q * UB) - c;
                RTPN_CHECK_PTR(kown + 3 * q + 1);
                const float4 k0 = kown[3 * q], k1 = kown[3 * q + 1];
                const float co = lds<S>(po, q * UB);
                const float ddy = lds<S>(py, q * UB) - co;
                RTPN_CHECK_PTR(koth + 3 * q + 2);
                const float4 k2 = koth[3 * q + 2];
                if constexpr (has_m) cur[am] = fmaf(k0.x, ddz, cur[am]);
                if constexpr (has_p) cur[ap] = fmaf(k0.y, ddz, cur[ap]);
                if constexpr (has_m) prev[am] = fmaf(k0.z, ddx, prev[am]);
                if constexpr (has_p) prev[ap] = fmaf(k0.w, ddx, prev[ap]);
                if constexpr (has_m) next[am] = fmaf(k1.x, ddx, next[am]);
                if constexpr (has_p) next[ap] = fmaf(k1.y, ddx, next[ap]);
                if constexpr (has_m) prev[am] = fmaf(k2.x, ddy, prev[am]);
                if constexpr (has_p) prev[ap] = fmaf(k2.y, ddy, prev[ap]);
                if constexpr (has_m) next[am] = fmaf(k2.z, ddy, next[am]);
                if constexpr (has_p) next[ap] = fmaf(k2.w, ddy, next[ap]);
            }
        }
    };
    auto chunk = [&](auto ci) {
        constexpr int C = decltype(ci)::value;
        static_for<kChunk>([&](auto ki) { slot(std::integral_constant<int, C * kChunk + decltype(ki)::value>{}); });
    };
    switch (fq / kChunk) { RTPN_CHUNK_CASES(chunk) }
}

// Finish target column M of type T (accumulators in prev) from its old values in the stage's
// target planes (at byte offset tgo for this cell) into global memory: FORWARD by Eq. (5),
// u' = alpha u - beta acc (the u_0 factors al0, be0, ga0 for slot 0 of column 0, cos type, class 0);
// ADJ_SOURCES lam' = alpha lam + acc / h (alpha = 1 when no factors are given).  tp: component q = 0 of the run at this cell, components V
// apart; only an active cell is stored.
template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EQ, int MODE>
RTPN_HD void finish_column(const unsigned char* buf, int tgo, int M, int T, S* tp, long long V, bool active,
                           float alpha, float beta, float al0, float be0, float ga0, float inv_h,
                           const float (&prev)[(N - A) / 2 + 1]) {
    using L = Layout<N, A, S, TX, TY, TZ, NB, EQ>;
    constexpr int UB = L::UB, NLA = (N - A) / 2 + 1;
    const bool u0 = A == 0 && M == 0 && T == 0;
    const int q0 = first_l(M, A) / 2;  // targets q = q0 .. NLA - 1 (l >= M)
    const unsigned char* ob = buf + tgo - q0 * UB;
    auto tslot = [&](auto qi) {
        constexpr int q = decltype(qi)::value;
        if constexpr (q < NLA) {
            const float old = lds<S>(ob, q * UB);
            float nv;
            if constexpr (MODE == ADJ_SOURCES)
                nv = fmaf(inv_h, prev[q], ((q == 0 && u0) ? al0 : alpha) * old);
            else if (q == 0)
                nv = u0 ? fmaf(al0, old, fmaf(-be0, prev[q], ga0)) : fmaf(alpha, old, -beta * prev[q]);
            else
                nv = fmaf(alpha, old, -beta * prev[q]);
            if (active) win::store<S>(tp + (long long)q * V, nv);
        }
    };
    switch (q0) { RTPN_SLOT_CASES(tslot) }
}

template <int N, int A, typename S, int TX, int TY, int TZ, int NB, int EQ, int MODE>
__device__ __forceinline__ void stage_kernel_body(const Args& a, unsigned char* smem) {
    using L = Layout<N, A, S, TX, TY, TZ, NB, EQ>;
    static_assert(N >= 1, "order N >= 1");
    static_assert((N + 2) / 2 <= kMaxSlots, "slot switch covers N <= 45");
    constexpr int B = 1 - A;
    constexpr int NLA = (N - A) / 2 + 1;   // class-A components of a run, at most
    constexpr int CELLS = L::CELLS;
    constexpr int REG = L::REG, ES = L::ES;
    constexpr int NST = N + 2;  // stage i: sources of column i (i <= N), targets of column i - 1
    const int cA0 = A == 0 ? 0 : class_size(N, 0);
    [[maybe_unused]] const int* colA = a.colstart + A * (N + 2);
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
        stage_producer<N, A, S, TX, TY, TZ, NB, EQ>(a, bufs, full0, empty0, total);
        return;
    }

    // ---- consumers: thread (T, cell) finishes the targets of type T in its cell.  Both types run
    // the same code: the type only selects regions, coupling-constant rows and the y direction.
    const int T = tid / CELLS, ctid = tid % CELLS;
    const int lx = ctid % TX, ly = (ctid / TX) % TY, lz = ctid / (TX * TY);
    const int tgo = L::TGTO + T * L::TGT_T + lz * REG + (ly * TX + lx) * ES;  // this cell's old target values

    // the three live target columns; their roles (prev, cur, next) rotate by one per stage
    float wa[NLA], wb[NLA], wc[NLA];

    TileGeo g{};
    bool active = false;
    long long cell = 0;
    Operands op{};                                     // operand offsets, fixed per tile
    float alE = 0.f, beE = 0.f, alO = 0.f, beO = 0.f;  // Eq. (5) factors of columns M even / odd
    float al0 = 0.f, be0 = 0.f, ga0 = 0.f;             // u_0 (class 0, type 0 only)

    // first local index of target column M in class A, advanced column by column (offA = colstart
    // of the column finished next)
    int offA = 0;
    unsigned tile = blockIdx.x;
    int b = 0;
    unsigned ph = 0;
    int s = 0, i = 0;

    // One stage: sweep source column i into prev (column i - 1), cur (i) and next (i + 1), finish
    // prev, and clear it (it is the next stage's `next`).  False if a wait ran out.
    auto stage = [&](float (&prev)[NLA], float (&cur)[NLA], float (&next)[NLA]) -> bool {
        if (i == 0) {  // new tile: geometry, operand offsets, factors, a cleared window
            if (s > 0) tile += gridDim.x;
            g = tile_geo<TX, TY, TZ, L::G>(a, tile);
            active = lx < g.wx && ly < g.wy && lz < g.wz;
            cell = ((long long)(g.z0 + lz) * a.ny + (g.y0 + ly)) * a.nx + (g.x0 + lx);
            op = operand_offsets<N, A, S, TX, TY, TZ, NB, EQ>(g, T, lx, ly, lz);
#pragma unroll
            for (int q = 0; q < NLA; ++q) prev[q] = cur[q] = next[q] = 0.f;
            if (active && (MODE == FORWARD || a.fac)) {  // ADJ_SOURCES: the alphas only, if asked
                // sub-grid slot of (l, M, T) in class A: x by (M, T), y by T, z by (A + M)
#pragma unroll
                for (int par = 0; par < 2; ++par) {
                    const int gx = ((par == 0) == (T == 0)) ? 0 : 1;
                    const int gz = ((A + par) & 1) == 0 ? 0 : 1;
                    const int gc = gx + 2 * T + 4 * gz;
                    const float al = __ldg(a.fac + (long long)(a.fac_ofs + 2 * gc) * V + cell);
                    // the pass folds 1/h into beta
                    const float be = __ldg(a.fac + (long long)(a.fac_ofs + 2 * gc + 1) * V + cell) * a.inv_h;
                    if (par == 0) {
                        alE = al;
                        beE = be;
                    } else {
                        alO = al;
                        beO = be;
                    }
                }
                if (A == 0 && T == 0) {
                    al0 = __ldg(a.fac + (long long)FAC_U0 * V + cell);
                    be0 = __ldg(a.fac + (long long)(FAC_U0 + 1) * V + cell) * a.inv_h;
                    ga0 = __ldg(a.fac + (long long)(FAC_U0 + 2) * V + cell);
                }
            } else if (MODE == ADJ_SOURCES) {
                alE = alO = al0 = 1.f;
            }
        }
        // target column i - 1 of type T is finished in this stage (the same for the whole warp); the
        // sweep and the finish run on every thread of the tile (a thread past the grid's edge works
        // on zero-filled or in-tile shared memory), only global memory accesses need an active cell
        const bool finw = i >= 1 && (T == 0 || i - 1 >= 1);

        if (!__all_sync(0xffffffffu, wait_phase(full0 + 8 * b, ph, a.wait_limit))) {
            if (lane == 0) atomicOr(a.status, STATUS_TIMEOUT);
            return false;
        }
        const unsigned char* buf = bufs + b * L::BUF;

        if (column_len(N, i, B) > 0) sweep_column<N, A, S, TX, TY, TZ, NB, EQ>(buf, op, T, i, prev, cur, next);
        if (finw) {
            const int M = i - 1;
            const float alpha = (M & 1) ? alO : alE, beta = (M & 1) ? beO : beE;
            const int q0 = first_l(M, A) / 2;
            (void)RTPN_SCHECK(offA == colA[M]);
            S* tp = reinterpret_cast<S*>(a.tgt) + (long long)(cA0 + offA + T * column_len(N, M, A) - q0) * V + cell;
            finish_column<N, A, S, TX, TY, TZ, NB, EQ, MODE>(buf, tgo, M, T, tp, V, active, alpha, beta, al0, be0,
                                                             ga0, a.inv_h, prev);
        }
        // the stage buffer is free once every lane of the warp is past its reads
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * b);
        if (++b == NB) {
            b = 0;
            ph ^= 1u;
        }
        // prev is done: it is the next stage's `next`
#pragma unroll
        for (int q = 0; q < NLA; ++q) prev[q] = 0.f;
        if (i >= 1) offA += ntypes(i - 1) * column_len(N, i - 1, A);
        if (i == NST - 1) offA = 0;  // tile done
        ++s;
        i = (i == NST - 1) ? 0 : i + 1;
        return true;
    };
    // the column loop unrolled by three: the window's roles rotate instead of its registers moving
    while (s < total) {
        if (!stage(wa, wb, wc) || s >= total) break;
        if (!stage(wb, wc, wa) || s >= total) break;
        if (!stage(wc, wa, wb)) break;
    }
}

}  // namespace stg
}  // namespace rtpn
