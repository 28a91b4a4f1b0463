// Host side of the TMA-staged kernels: variant registry, tensor maps, coupling tables, launch.
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "stage_impl.cuh"
#include "stage_variants.h"

namespace rtpn {
namespace stg {

#define RTPN_SDECL(n, x, y, z, b, e)                                                                 \
    int stage_launch_##n##_##x##_##y##_##z##_##b##_##e(int, int, int, const Args&, int, cudaStream_t);  \
    int stage_smem_##n##_##x##_##y##_##z##_##b##_##e(int, int);                                          \
    void stage_geom_##n##_##x##_##y##_##z##_##b##_##e(int, int*);
RTPN_STAGE_VARIANTS(RTPN_SDECL)
#undef RTPN_SDECL

struct Variant {
    int N, tx, ty, tz, depth;
    int (*launch)(int, int, int, const Args&, int, cudaStream_t);  // (cls, precision, mode, ...)
    int (*smem)(int, int);
    void (*geom)(int, int*);  // (precision, {maps per kind, box length step, x group width, x group rows})
};
#define RTPN_SENTRY(n, x, y, z, b, e)                                                                \
    Variant{n, x, y, z, b, stage_launch_##n##_##x##_##y##_##z##_##b##_##e,                           \
            stage_smem_##n##_##x##_##y##_##z##_##b##_##e, stage_geom_##n##_##x##_##y##_##z##_##b##_##e},
static const Variant kVariants[] = {RTPN_STAGE_VARIANTS(RTPN_SENTRY)};
#undef RTPN_SENTRY

// a variant is usable for a storage precision if its stage ring fits shared memory
static bool fits(const Variant& v, int precision) { return v.smem(0, precision) > 0 && v.smem(1, precision) > 0; }

// first compiled variant of order N with this tile (0 = any) and depth (0 = any) that fits
static const Variant* find(int N, int tx, int ty, int tz, int depth, int precision) {
    for (const auto& v : kVariants)
        if (v.N == N && (tx == 0 || (v.tx == tx && v.ty == ty && v.tz == tz)) &&
            (depth == 0 || v.depth == depth) && fits(v, precision))
            return &v;
    return nullptr;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

static bool make_map(CUtensorMap* m, void* base, int precision, const rtpn::Geom& g, int nc, int bx, int by,
                     int bz, int bc) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t es = precision == RTPN_BF16 ? 2 : 4;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)nc};
    const cuuint64_t strides[3] = {g.nx * es, (cuuint64_t)g.nx * g.ny * es, (cuuint64_t)g.V * es};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, (cuuint32_t)bc};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(m, precision == RTPN_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The tensor maps of one array for a variant (kinds MAP_PLANE, MAP_YROW, MAP_XGRP, each for box
// lengths E = eq, 2 eq, ..., nmap eq; see stage_impl.cuh) into out[0 .. kinds * nmap); kinds = 1 builds
// the plane maps only (target arrays).
static bool make_maps(CUtensorMap* out, void* base, int precision, const rtpn::Geom& g, int nc, const Variant& v,
                      int kinds) {
    int geo[4];
    v.geom(precision, geo);
    const int nmap = geo[0], eq = geo[1], xw = geo[2], ry = geo[3];
    for (int j = 0; j < nmap; ++j) {
        const int e = eq * (j + 1);
        if (!make_map(&out[MAP_PLANE * nmap + j], base, precision, g, nc, v.tx, v.ty, 1, e)) return false;
        if (kinds > 1 && (!make_map(&out[MAP_YROW * nmap + j], base, precision, g, nc, v.tx, 1, v.tz, e) ||
                          !make_map(&out[MAP_XGRP * nmap + j], base, precision, g, nc, xw, ry, v.tz, e)))
            return false;
    }
    return true;
}

static int nmaps_of(const Variant& v, int precision) {
    int geo[4];
    v.geom(precision, geo);
    return geo[0];
}

}  // namespace stg

// device tensor-map slots of a context: forward (all kinds), adjoint w (all kinds), adjoint lam (plane)
static constexpr int stage_maps_capacity = (2 * stg::MAP_KINDS + 1) * stg::kMaxSlots;

bool stage_supported(int N, int precision, int nx) {
    if (precision == RTPN_FP64 || !stg::find(N, 0, 0, 0, 0, precision)) return false;
    const int hx = precision == RTPN_BF16 ? 8 : 4;  // 16-byte rows for the tensor maps
    return nx % hx == 0;
}

bool stage_has_tile(int N, int tx, int ty, int tz, int depth, int precision) {
    return stg::find(N, tx, ty, tz, depth, precision) != nullptr;
}

int stage_prepare(rtpn_ctx* ctx, int tx, int ty, int tz, int depth) {
    const stg::Variant* v = stg::find(ctx->N, tx, ty, tz, depth, ctx->prec);
    if (!v) return (int)cudaErrorNotSupported;
    // default (no tile given): the first listed variant whose width divides nx, else the first one
    if (tx == 0)
        for (const auto& w : stg::kVariants)
            if (w.N == ctx->N && (depth == 0 || w.depth == depth) && ctx->g.nx % w.tx == 0 &&
                stg::fits(w, ctx->prec)) {
                v = &w;
                break;
            }
    const int N = ctx->N;
    // the tensor maps live in device global memory (64-byte aligned) and the kernel reads them from
    // there: tile planes / z halo plane, y halo row and x halo group, each for every box length
    const int nmap = stg::nmaps_of(*v, ctx->prec);
    if (nmap <= 0 || nmap > stg::kMaxSlots) return (int)cudaErrorInvalidValue;
    std::vector<CUtensorMap> maps((size_t)stg::MAP_KINDS * nmap);
    if (!stg::make_maps(maps.data(), ctx->u, ctx->prec, ctx->g, ctx->md.nc, *v, stg::MAP_KINDS))
        return (int)cudaErrorInvalidValue;
    if (!ctx->stage_maps_dev) {
        // the forward's maps, then room for the adjoint's (all kinds over w, plane maps over lam)
        cudaError_t err = cudaMalloc(&ctx->stage_maps_dev, stage_maps_capacity * sizeof(CUtensorMap));
        if (err != cudaSuccess) return (int)err;
    }
    {
        cudaError_t err = cudaMemcpy(ctx->stage_maps_dev, maps.data(), maps.size() * sizeof(CUtensorMap),
                                     cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return (int)err;
        ctx->stage_adj_lam = ctx->stage_adj_w = nullptr;  // the adjoint's maps follow the tile
    }
    if (!ctx->stage_mem) {
        std::vector<int> col;
        std::vector<float> tab[2];
        if (!stg::coupling_tables(ctx->md, ctx->g.h / ctx->g.hy, ctx->g.h / ctx->g.hz, tab, &col))
            return (int)cudaErrorInvalidValue;
        const size_t b0 = tab[0].size() * 4, b1 = tab[1].size() * 4, b2 = col.size() * 4;
        cudaError_t err = cudaMalloc(&ctx->stage_mem, b0 + b1 + b2);
        if (err != cudaSuccess) return (int)err;
        char* m = (char*)ctx->stage_mem;
        cudaMemcpy(m, tab[0].data(), b0, cudaMemcpyHostToDevice);
        cudaMemcpy(m + b0, tab[1].data(), b1, cudaMemcpyHostToDevice);
        err = cudaMemcpy(m + b0 + b1, col.data(), b2, cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return (int)err;
        ctx->stage_tab_bytes[0] = b0;
        ctx->stage_tab_bytes[1] = b1;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
    ctx->stage_variant = (int)(v - stg::kVariants);
    ctx->tx = v->tx;
    ctx->ty = v->ty;
    ctx->tz = v->tz;
    ctx->depth = v->depth;
    ctx->tile_from_stage = true;
    return 0;
}

// the compiled (tile, depth) choices of order N, for the tuner
int stage_variants_of(int N, int precision, int* tiles, int max) {
    int n = 0;
    for (const auto& v : stg::kVariants)
        if (v.N == N && stg::fits(v, precision) && n < max) {
            tiles[4 * n] = v.tx;
            tiles[4 * n + 1] = v.ty;
            tiles[4 * n + 2] = v.tz;
            tiles[4 * n + 3] = v.depth;
            ++n;
        }
    return n;
}

// The launch fields every mode shares: geometry, the tile walk, the coupling table of a forward
// pass on class coef_cls (its sources are the other class), the status word and the wait limit.
static bool base_args(const rtpn_ctx* ctx, const stg::Variant& v, int coef_cls, stg::Args* out) {
    stg::Args a{};
    const char* m = (const char*)ctx->stage_mem;
    a.coefcol = (const float*)(coef_cls == 0 ? m : m + ctx->stage_tab_bytes[0]);
    a.colstart = (const int*)(m + ctx->stage_tab_bytes[0] + ctx->stage_tab_bytes[1]);
    a.V = ctx->g.V;
    a.nx = ctx->g.nx;
    a.ny = ctx->g.ny;
    a.nz = ctx->g.nz;
    a.bc = ctx->g.bc;
    a.inv_h = (float)(1.0 / ctx->g.h);
    a.ntx = (a.nx + v.tx - 1) / v.tx;
    a.nty = (a.ny + v.ty - 1) / v.ty;
    a.ntz = (a.nz + v.tz - 1) / v.tz;
    a.tiles = (long long)a.ntx * a.nty * a.ntz;
    if (a.tiles * (ctx->N + 2) >= (1ll << 31)) return false;
    // z chunk of the tile walk: the ~one tile per SM at work at a time then spans about as many
    // tile rows in y as layers in z, across the whole x extent
    const double side = std::sqrt((double)(ctx->sms > 0 ? ctx->sms : 1) / a.ntx);
    const int kz = (int)(side + 0.5);
    a.kz = kz < 1 ? 1 : (kz > a.ntz ? a.ntz : kz);
    a.nc = ctx->md.nc;
    a.status = ctx->status;
    a.wait_limit = (unsigned)STAGE_WAIT_LIMIT;
    a.skip_stage = -1;
    *out = a;
    return true;
}

// a forward pass on class cls: sources through src_maps, old targets through the plane maps
// tgt_maps, new targets stored into out (all three may be the context's state)
static int launch_pass(rtpn_ctx* ctx, int cls, int fac_ofs, const CUtensorMap* src_maps,
                       const CUtensorMap* tgt_maps, void* out, cudaStream_t st, long long skip_stage,
                       long long wait_limit) {
    if (ctx->stage_variant < 0) return (int)cudaErrorNotSupported;
    const stg::Variant& v = stg::kVariants[ctx->stage_variant];
    stg::Args a;
    if (!base_args(ctx, v, cls, &a)) return (int)cudaErrorInvalidValue;
    a.tgt = out;
    a.fac = (const float*)ctx->fac;
    a.fac_ofs = fac_ofs;
    a.maps = src_maps;
    a.tmap = tgt_maps;
    a.src_c0 = cls == 1 ? 0 : ctx->md.ne;  // the source class is the other one
    a.wait_limit = (unsigned)(wait_limit > 0xffffffffll ? 0xffffffffll : wait_limit);
    a.skip_stage = skip_stage;
    return v.launch(cls, ctx->prec, stg::FORWARD, a, ctx->sms, st);
}

int launch_stage(rtpn_ctx* ctx, int cls, int fac_ofs, cudaStream_t st, long long skip_stage,
                 long long wait_limit) {
    const CUtensorMap* maps = (const CUtensorMap*)ctx->stage_maps_dev;  // sources and targets: the state
    return launch_pass(ctx, cls, fac_ofs, maps, maps, ctx->u, st, skip_stage, wait_limit);
}

int launch_stage_between(rtpn_ctx* ctx, int cls, int fac_ofs, const void* src_maps, const void* tgt_maps,
                         void* out, cudaStream_t st) {
    if (ctx->prec != RTPN_FP32) return (int)cudaErrorNotSupported;
    return launch_pass(ctx, cls, fac_ofs, (const CUtensorMap*)src_maps, (const CUtensorMap*)tgt_maps, out, st,
                       -1, STAGE_WAIT_LIMIT);
}

size_t stage_maps_bytes(const rtpn_ctx* ctx) {
    if (ctx->stage_variant < 0) return 0;
    return (size_t)stg::MAP_KINDS * stg::nmaps_of(stg::kVariants[ctx->stage_variant], ctx->prec) *
           sizeof(CUtensorMap);
}

int stage_maps_for(rtpn_ctx* ctx, const void* state, void* maps_dev) {
    if (ctx->stage_variant < 0 || ctx->prec != RTPN_FP32) return (int)cudaErrorNotSupported;
    const stg::Variant& v = stg::kVariants[ctx->stage_variant];
    std::vector<CUtensorMap> maps((size_t)stg::MAP_KINDS * stg::nmaps_of(v, RTPN_FP32));
    if (!stg::make_maps(maps.data(), const_cast<void*>(state), RTPN_FP32, ctx->g, ctx->md.nc, v, stg::MAP_KINDS))
        return (int)cudaErrorInvalidValue;
    return (int)cudaMemcpy(maps_dev, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
}

int launch_stage_adjoint_sources(rtpn_ctx* ctx, int tgt_cls, float* lam, const float* w, int w_planes,
                                 int fac_ofs, cudaStream_t st) {
    if (ctx->stage_variant < 0 || ctx->prec != RTPN_FP32) return (int)cudaErrorNotSupported;
    const stg::Variant& v = stg::kVariants[ctx->stage_variant];
    // tensor maps over w (every source box kind) and over lam (target planes), rebuilt when the
    // arrays change (once per adjoint call); they follow the forward maps
    const int nmap = stg::nmaps_of(v, RTPN_FP32);
    CUtensorMap* dev = (CUtensorMap*)ctx->stage_maps_dev + stg::MAP_KINDS * nmap;
    if (ctx->stage_adj_lam != lam || ctx->stage_adj_w != w) {
        std::vector<CUtensorMap> maps((size_t)(stg::MAP_KINDS + 1) * nmap);
        if (!stg::make_maps(maps.data(), const_cast<float*>(w), RTPN_FP32, ctx->g, w_planes, v, stg::MAP_KINDS) ||
            !stg::make_maps(maps.data() + stg::MAP_KINDS * nmap, lam, RTPN_FP32, ctx->g, ctx->md.nc, v, 1))
            return (int)cudaErrorInvalidValue;
        cudaError_t err = cudaMemcpy(dev, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return (int)err;
        ctx->stage_adj_lam = lam;
        ctx->stage_adj_w = w;
    }
    // the coupling table of a forward pass on the target class: its sources are the other class
    stg::Args a;
    if (!base_args(ctx, v, tgt_cls, &a)) return (int)cudaErrorInvalidValue;
    a.tgt = lam;
    a.fac = fac_ofs >= 0 ? (const float*)ctx->fac : nullptr;  // lam_B <- alpha_B lam_B folded in
    a.fac_ofs = fac_ofs >= 0 ? fac_ofs : 0;
    a.maps = dev;
    a.tmap = dev + stg::MAP_KINDS * nmap;
    a.src_c0 = 0;  // w holds only the source class, in its local order
    a.nc = w_planes;
    return v.launch(tgt_cls, RTPN_FP32, stg::ADJ_SOURCES, a, ctx->sms, st);
}

}  // namespace rtpn
