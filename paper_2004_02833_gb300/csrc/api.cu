// The C ABI of include/rtpn.h: context life cycle, data movement and the step schedule.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <string>
#include <utility>

#include "rtpn_internal.h"

using namespace rtpn;

namespace {

thread_local std::string g_create_err;

int fail(rtpn_ctx* ctx, int code, const std::string& msg) {
    if (ctx)
        ctx->err = msg;
    else
        g_create_err = msg;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? RTPN_ENOMEM : RTPN_ECUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

#define CHECK_LAUNCH(ctx)                                                                        \
    do {                                                                                         \
        cudaError_t e_ = cudaGetLastError();                                                     \
        if (e_ != cudaSuccess)                                                                   \
            return fail(ctx, RTPN_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

size_t dtype_size(int dtype) { return dtype == RTPN_DTYPE_F64 ? 8 : 4; }

bool valid_dtype(int d) { return d == RTPN_DTYPE_F64 || d == RTPN_DTYPE_F32; }
bool valid_where(int w) { return w == RTPN_HOST || w == RTPN_DEVICE; }

// typed dispatch on the storage precision
template <typename Fn>
void with_storage(int prec, Fn&& fn) {
    if (prec == RTPN_FP64)
        fn((double*)nullptr);
    else if (prec == RTPN_FP32)
        fn((float*)nullptr);
    else
        fn((__nv_bfloat16*)nullptr);
}

// convert `n` values of caller dtype at device pointer `in` into storage at `out`
int convert_in(rtpn_ctx* ctx, const void* in, int dtype, void* out, long long n) {
    with_storage(ctx->prec, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (dtype == RTPN_DTYPE_F64)
            launch_convert<double, S>((const double*)in, (S*)out, n, ctx->stream);
        else
            launch_convert<float, S>((const float*)in, (S*)out, n, ctx->stream);
    });
    CHECK_LAUNCH(ctx);
    return RTPN_OK;
}

int convert_out(rtpn_ctx* ctx, const void* in, void* out, int dtype, long long n) {
    with_storage(ctx->prec, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (dtype == RTPN_DTYPE_F64)
            launch_convert<S, double>((const S*)in, (double*)out, n, ctx->stream);
        else
            launch_convert<S, float>((const S*)in, (float*)out, n, ctx->stream);
    });
    CHECK_LAUNCH(ctx);
    return RTPN_OK;
}

bool same_type(int prec, int dtype) {
    return (prec == RTPN_FP64 && dtype == RTPN_DTYPE_F64) ||
           (prec == RTPN_FP32 && dtype == RTPN_DTYPE_F32);
}

void* comp_ptr(rtpn_ctx* ctx, int internal) {
    return (char*)ctx->u + (size_t)internal * ctx->g.V * ctx->elem;
}

int put_component(rtpn_ctx* ctx, int abi, const void* src, int dtype, int where) {
    const long long V = ctx->g.V;
    void* dst = comp_ptr(ctx, ctx->md.internal_of_abi[abi]);
    const size_t bytes = (size_t)V * dtype_size(dtype);
    if (same_type(ctx->prec, dtype)) {
        CUDA_TRY(ctx, cudaMemcpyAsync(dst, src, bytes,
                                      where == RTPN_HOST ? cudaMemcpyHostToDevice
                                                         : cudaMemcpyDeviceToDevice,
                                      ctx->stream));
        return RTPN_OK;
    }
    const void* dev_src = src;
    if (where == RTPN_HOST) {
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->staging, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
        dev_src = ctx->staging;
    }
    return convert_in(ctx, dev_src, dtype, dst, V);
}

int take_component(rtpn_ctx* ctx, int abi, void* dst, int dtype, int where) {
    const long long V = ctx->g.V;
    const void* src = comp_ptr(ctx, ctx->md.internal_of_abi[abi]);
    const size_t bytes = (size_t)V * dtype_size(dtype);
    if (same_type(ctx->prec, dtype)) {
        CUDA_TRY(ctx, cudaMemcpyAsync(dst, src, bytes,
                                      where == RTPN_HOST ? cudaMemcpyDeviceToHost
                                                         : cudaMemcpyDeviceToDevice,
                                      ctx->stream));
        return RTPN_OK;
    }
    if (where == RTPN_DEVICE) return convert_out(ctx, src, dst, dtype, V);
    int rc = convert_out(ctx, src, ctx->staging, dtype, V);
    if (rc) return rc;
    CUDA_TRY(ctx, cudaMemcpyAsync(dst, ctx->staging, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    return RTPN_OK;
}

// ------------------------------------------------------------------ step schedule
int run_pass(rtpn_ctx* ctx, int cls, int fac_ofs, cudaStream_t st) {
    if (ctx->active_kernel == RTPN_KERNEL_STAGE) {
        int rc = launch_stage(ctx, cls, fac_ofs, st, -1, STAGE_WAIT_LIMIT);
        if (rc) return fail(ctx, RTPN_ECUDA, std::string("staged kernel: ") +
                                                 cudaGetErrorString((cudaError_t)rc));
    } else if (ctx->active_kernel == RTPN_KERNEL_WINDOW || ctx->active_kernel == RTPN_KERNEL_FUSED) {
        WindowLaunch w;
        w.u = ctx->u;
        w.fac = (const float*)ctx->fac;
        w.g = ctx->g;
        w.cls = cls;
        w.aniso = ctx->scat != nullptr;
        w.fac_ofs = w.aniso && fac_ofs == FAC_HALF ? aniso_half_ofs(ctx->N) : fac_ofs;
        const bool own_tile = ctx->active_kernel == RTPN_KERNEL_WINDOW;
        w.tx = own_tile ? ctx->tx : 0;
        w.ty = own_tile ? ctx->ty : 0;
        w.tz = own_tile ? ctx->tz : 0;
        int rc = launch_window(ctx->N, ctx->prec, w, st);
        if (rc) return fail(ctx, RTPN_ECUDA, std::string("window kernel: ") +
                                                 cudaGetErrorString((cudaError_t)rc));
    } else if (ctx->prec == RTPN_FP64) {
        if (ctx->scat && fac_ofs == FAC_HALF) fac_ofs = aniso_half_ofs(ctx->N);
        launch_substep_generic<double, double>((double*)ctx->u, (const double*)ctx->fac,
                                               ctx->tab64[cls], ctx->g, fac_ofs, st);
    } else if (ctx->prec == RTPN_FP32) {
        if (ctx->scat && fac_ofs == FAC_HALF) fac_ofs = aniso_half_ofs(ctx->N);
        launch_substep_generic<float, float>((float*)ctx->u, (const float*)ctx->fac,
                                             ctx->tab32[cls], ctx->g, fac_ofs, st);
    } else {
        if (ctx->scat && fac_ofs == FAC_HALF) fac_ofs = aniso_half_ofs(ctx->N);
        launch_substep_generic<__nv_bfloat16, float>((__nv_bfloat16*)ctx->u,
                                                     (const float*)ctx->fac, ctx->tab32[cls],
                                                     ctx->g, fac_ofs, st);
    }
    CHECK_LAUNCH(ctx);
    return RTPN_OK;
}

// One fused pass (even full step, odd step with factors fac_odd) from state x into state y.
int fused_pass(rtpn_ctx* ctx, const void* x, void* y, int fac_odd, cudaStream_t st) {
    FusedLaunch f;
    f.x = x;
    f.y = y;
    f.fac = (const float*)ctx->fac;
    f.g = ctx->g;
    f.fac_odd = fac_odd;
    f.zc = ctx->tz;
    int rc = launch_fused(ctx->N, ctx->prec, f, st);
    if (rc) return fail(ctx, RTPN_ECUDA, std::string("fused kernel: ") + cudaGetErrorString((cudaError_t)rc));
    return RTPN_OK;
}

void* other_buffer(const rtpn_ctx* ctx, const void* cur) { return cur == ctx->u ? ctx->u_alt : ctx->u; }

// `pairs` fused passes alternating between the two buffers, starting from state `from`; the state
// ends in `from` for an even count and in the other buffer for an odd one.
int enqueue_fused(rtpn_ctx* ctx, int pairs, void* from, cudaStream_t st) {
    void* x = from;
    for (int p = 0; p < pairs; ++p) {
        void* y = other_buffer(ctx, x);
        int rc = fused_pass(ctx, x, y, FAC_FULL, st);
        if (rc) return rc;
        x = y;
    }
    return RTPN_OK;
}

int enqueue_pairs(rtpn_ctx* ctx, int pairs, bool fused, cudaStream_t st) {
    if (fused) return enqueue_fused(ctx, pairs, ctx->u, st);
    for (int p = 0; p < pairs; ++p) {
        int rc = run_pass(ctx, 0, FAC_FULL, st);
        if (rc) return rc;
        rc = run_pass(ctx, 1, FAC_FULL, st);
        if (rc) return rc;
    }
    return RTPN_OK;
}

void drop_graphs(rtpn_ctx* ctx) {
    for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
}

// (even, odd) full-step pairs, replayed from cached graphs of 64 / 8 / 1 pairs.  Fused passes
// alternate between the two state buffers: their graphs are keyed by which buffer they start from
// (the buffer addresses are fixed for the life of the context) and ctx->u follows the state.
// `fused` = false runs the two-pass schedule (also with RTPN_KERNEL_FUSED active).
int launch_pairs(rtpn_ctx* ctx, int pairs, bool fused) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CUDA_TRY(ctx, cudaStreamIsCapturing(ctx->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        int rc = enqueue_pairs(ctx, pairs, fused, ctx->stream);
        if (!rc && fused && (pairs & 1)) std::swap(ctx->u, ctx->u_alt);
        return rc;
    }
    const int sizes[3] = {64, 8, 1};
    for (int s : sizes) {
        while (pairs >= s) {
            // key: pair count, plus 1 << 20 for fused graphs starting from the second buffer
            const int key = fused ? s + (1 << 16) + (ctx->u == ctx->u_home ? 0 : 1 << 20) : s;
            auto it = ctx->graphs.find(key);
            if (it == ctx->graphs.end()) {
                cudaGraph_t graph = nullptr;
                CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->own, cudaStreamCaptureModeThreadLocal));
                int rc = enqueue_pairs(ctx, s, fused, ctx->own);
                cudaError_t e = cudaStreamEndCapture(ctx->own, &graph);
                if (rc) {
                    if (graph) cudaGraphDestroy(graph);
                    return rc;
                }
                if (e != cudaSuccess)
                    return fail(ctx, RTPN_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
                cudaGraphExec_t exec = nullptr;
                e = cudaGraphInstantiate(&exec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess)
                    return fail(ctx, RTPN_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
                it = ctx->graphs.emplace(key, exec).first;
            }
            CUDA_TRY(ctx, cudaGraphLaunch(it->second, ctx->stream));
            if (fused && (s & 1)) std::swap(ctx->u, ctx->u_alt);
            pairs -= s;
        }
    }
    return RTPN_OK;
}

HostTable host_table(const Model& md, int cls, const Geom& g, bool aniso) {
    HostTable t;
    t.a0 = cls == 0 ? 0 : md.ne;
    t.na = cls == 0 ? md.ne : md.no;
    t.row.push_back(0);
    // md.nz is sorted by row (interface index); targets come in internal order, so index rows first
    std::vector<size_t> first(md.nc + 1, md.nz.size());
    for (size_t q = md.nz.size(); q-- > 0;) first[md.nz[q].a] = q;
    for (int i = t.a0; i < t.a0 + t.na; ++i) {
        const int a = md.abi_of_internal[i];
        const Component& ca = md.comp[a];
        for (size_t q = first[a]; q < md.nz.size() && md.nz[q].a == a; ++q) {
            const Coupling& e = md.nz[q];
            const bool upper = ca.slot[e.axis] == 2;  // target on a 2-slot reads cells i, i+1
            t.src.push_back(md.internal_of_abi[e.b]);
            t.code.push_back(e.axis * 2 + (upper ? 1 : 0));
            t.coef.push_back((upper ? 1.0 : -1.0) * e.v / axis_h(g, e.axis));
        }
        t.row.push_back((int)t.src.size());
        t.fplane.push_back(a == 0 ? FAC_U0
                                  : aniso ? aniso_plane(md.N, slot_code(ca.slot), ca.l) : 2 * slot_code(ca.slot));
    }
    return t;
}

// upload both classes' tables into one allocation (ints, then doubles, then floats)
int upload_tables(rtpn_ctx* ctx) {
    const bool aniso = ctx->scat != nullptr;
    HostTable t[2] = {host_table(ctx->md, 0, ctx->g, aniso), host_table(ctx->md, 1, ctx->g, aniso)};
    size_t bytes = 0;
    for (auto& x : t)
        bytes += (x.row.size() + x.src.size() + x.code.size() + x.fplane.size()) * sizeof(int) +
                 x.coef.size() * (sizeof(double) + sizeof(float)) + 64;
    CUDA_TRY(ctx, cudaMalloc(&ctx->table_mem, bytes));
    std::vector<char> host(bytes, 0);
    size_t off = 0;
    auto put = [&](const void* src, size_t n) {
        off = (off + 7) & ~size_t(7);
        std::memcpy(host.data() + off, src, n);
        size_t at = off;
        off += n;
        return (char*)ctx->table_mem + at;
    };
    for (int c = 0; c < 2; ++c) {
        auto& x = t[c];
        std::vector<float> cf(x.coef.begin(), x.coef.end());
        const int* row = (const int*)put(x.row.data(), x.row.size() * sizeof(int));
        const int* src = (const int*)put(x.src.data(), x.src.size() * sizeof(int));
        const int* code = (const int*)put(x.code.data(), x.code.size() * sizeof(int));
        const int* fp = (const int*)put(x.fplane.data(), x.fplane.size() * sizeof(int));
        const double* c64 = (const double*)put(x.coef.data(), x.coef.size() * sizeof(double));
        const float* c32 = (const float*)put(cf.data(), cf.size() * sizeof(float));
        ctx->tab64[c] = {row, src, c64, code, fp, x.a0, x.na};
        ctx->tab32[c] = {row, src, c32, code, fp, x.a0, x.na};
    }
    CUDA_TRY(ctx, cudaMemcpy(ctx->table_mem, host.data(), bytes, cudaMemcpyHostToDevice));
    return RTPN_OK;
}

void release(rtpn_ctx* ctx) {
    drop_graphs(ctx);
    if (ctx->u) cudaFree(ctx->u);
    if (ctx->u_alt) cudaFree(ctx->u_alt);
    ctx->u_alt = ctx->u_home = nullptr;
    if (ctx->fac) cudaFree(ctx->fac);
    if (ctx->scat) cudaFree(ctx->scat);
    ctx->scat = nullptr;
    if (ctx->table_mem) cudaFree(ctx->table_mem);
    if (ctx->partial) cudaFree(ctx->partial);
    if (ctx->counter) cudaFree(ctx->counter);
    if (ctx->staging) cudaFree(ctx->staging);
    if (ctx->status) cudaFree(ctx->status);
    if (ctx->media) cudaFree(ctx->media);
    ctx->media = nullptr;
    if (ctx->stage_mem) cudaFree(ctx->stage_mem);
    if (ctx->stage_maps_dev) cudaFree(ctx->stage_maps_dev);
    ctx->stage_maps_dev = nullptr;
    if (ctx->adj_ws) cudaFree(ctx->adj_ws);
    ctx->adj_ws = nullptr;
    ctx->adj_ws_bytes = 0;
    for (long long& k : ctx->adj_maps_key) k = -1;
    ctx->status = nullptr;
    ctx->stage_mem = nullptr;
    if (ctx->own) cudaStreamDestroy(ctx->own);
    ctx->u = ctx->fac = ctx->table_mem = ctx->staging = nullptr;
    ctx->partial = nullptr;
    ctx->counter = nullptr;
    ctx->own = nullptr;
}

// Automatic selection: the staged kernel where it is compiled for (N, precision), N >= kStageMinN
// and nx gives 16-byte rows, else the register-window kernel, else the generic one.  Below
// kStageMinN the unrolled window body is small enough for the instruction cache and the staged
// kernel's per-column-stage overhead dominates its few components per column (P7 128^3 FP32 on a
// GB300: 0.41 ms per step with the window kernel, 0.92 with the staged one; P15: 2.16 and 2.02).
constexpr bool kStageInAuto = true;
constexpr int kStageMinN = 15;

int choose_kernel(rtpn_ctx* ctx) {
    int k = ctx->kernel;
    const bool cubic = cubic_cells(ctx->g);
    if (ctx->scat) {
        // per-order factors: the generic kernel's per-target plane table, or the window kernel's
        // anisotropic form (N <= 15), which reads each target's planes at its finish
        const bool win_aniso = window_supported(ctx->N, ctx->prec) && window_extended(ctx->N);
        if (k == RTPN_KERNEL_AUTO) k = win_aniso ? RTPN_KERNEL_WINDOW : RTPN_KERNEL_GENERIC;
        if (k != RTPN_KERNEL_GENERIC && !(k == RTPN_KERNEL_WINDOW && win_aniso))
            return fail(ctx, RTPN_EUNSUPPORTED,
                        "anisotropic scattering runs on the generic kernel and the window kernel up to N = 15");
    }
    // the window kernel takes non-cubic cells up to N = 15 (scaled y and z differences); the fused
    // kernel takes cubic cells only
    const bool win_ok = window_supported(ctx->N, ctx->prec) && (cubic || window_extended(ctx->N));
    if (k == RTPN_KERNEL_AUTO) {
        const bool tile_set = ctx->tx || ctx->ty || ctx->tz;
        if (kStageInAuto && (ctx->N >= kStageMinN || !win_ok) &&
            stage_supported(ctx->N, ctx->prec, ctx->g.nx) &&
            (!tile_set || stage_has_tile(ctx->N, ctx->tx, ctx->ty, ctx->tz, ctx->depth, ctx->prec)))
            k = RTPN_KERNEL_STAGE;
        else
            k = win_ok ? RTPN_KERNEL_WINDOW : RTPN_KERNEL_GENERIC;
    }
    // a tile the staged kernel chose is no request for another kernel (its shape need not even be a
    // valid window tile): the other kernels start from their defaults
    if (k != RTPN_KERNEL_STAGE && ctx->tile_from_stage) {
        ctx->tx = ctx->ty = ctx->tz = 0;
        ctx->depth = 0;
        ctx->tile_from_stage = false;
    }
    if (!cubic && k == RTPN_KERNEL_FUSED)
        return fail(ctx, RTPN_EUNSUPPORTED, "the fused kernel takes cubic cells only");
    if (!cubic && k == RTPN_KERNEL_WINDOW && !window_extended(ctx->N))
        return fail(ctx, RTPN_EUNSUPPORTED, "the window kernel takes non-cubic cells up to N = 15 only");
    if (k == RTPN_KERNEL_STAGE) {
        if (!stage_supported(ctx->N, ctx->prec, ctx->g.nx))
            return fail(ctx, RTPN_EUNSUPPORTED,
                        "staged kernel not compiled for this N/precision or nx*elem not 16-byte rows");
        if (!stage_has_tile(ctx->N, ctx->tx, ctx->ty, ctx->tz, ctx->depth, ctx->prec))
            return fail(ctx, RTPN_EUNSUPPORTED, "no staged kernel compiled for this tile / stage depth");
        int rc = stage_prepare(ctx, ctx->tx, ctx->ty, ctx->tz, ctx->depth);
        if (rc) return fail(ctx, RTPN_ECUDA, std::string("staged kernel set-up: ") +
                                                 cudaGetErrorString((cudaError_t)rc));
    }
    if (k == RTPN_KERNEL_WINDOW) {
        if (!window_supported(ctx->N, ctx->prec))
            return fail(ctx, RTPN_EUNSUPPORTED, "window kernel not compiled for this N/precision");
        int rc = window_prepare(ctx->md, ctx->g.h, ctx->prec);
        if (rc) return fail(ctx, RTPN_ECUDA, std::string("window constants: ") +
                                                 cudaGetErrorString((cudaError_t)rc));
    }
    if (k == RTPN_KERNEL_FUSED) {
        // a batch keeps each instance's state pointer in its launch items; the fused kernel moves it
        if (ctx->batch_member)
            return fail(ctx, RTPN_EUNSUPPORTED, "batch instances keep their state in one buffer");
        if (!fused_supported(ctx->N, ctx->prec) || !window_supported(ctx->N, ctx->prec))
            return fail(ctx, RTPN_EUNSUPPORTED, "fused kernel not compiled for this N/precision");
        int rc = fused_prepare(ctx->md, ctx->prec);
        if (!rc) rc = window_prepare(ctx->md, ctx->g.h, ctx->prec);
        if (rc) return fail(ctx, RTPN_ECUDA, std::string("fused kernel constants: ") +
                                                 cudaGetErrorString((cudaError_t)rc));
        if (!ctx->u_alt) {
            cudaError_t e = cudaMalloc(&ctx->u_alt, (size_t)ctx->md.nc * ctx->g.V * ctx->elem);
            if (e != cudaSuccess) {
                ctx->u_alt = nullptr;
                cudaGetLastError();
                return fail(ctx, RTPN_ENOMEM, "second state buffer of the fused kernel");
            }
        }
    }
    if (k != ctx->active_kernel) drop_graphs(ctx);
    ctx->active_kernel = k;
    return RTPN_OK;
}

}  // namespace

namespace rtpn {
// Message for rtpn_last_error(NULL) from entry points that take no context.
void note_error(const std::string& msg) { g_create_err = msg; }
}  // namespace rtpn

// ==================================================================== C ABI
extern "C" {

int rtpn_version(void) { return 100; }

const char* rtpn_strerror(int code) {
    switch (code) {
        case RTPN_OK: return "ok";
        case RTPN_EINVAL: return "invalid argument";
        case RTPN_ECFL: return "time step violates dt < min(h)/3";
        case RTPN_ENOMEM: return "device allocation failed";
        case RTPN_ECUDA: return "CUDA error";
        case RTPN_ETIMEOUT: return "bounded device wait expired";
        case RTPN_ENONFINITE: return "non-finite values in the state";
        case RTPN_EUNSUPPORTED: return "not compiled into this library";
        case RTPN_ESTATE: return "call out of order";
        default: return "unknown status";
    }
}

int rtpn_component_info(int N, int c, int* l, int* m, int slots[3], int* cls) {
    if (N < 0 || N > 63 || c < 0 || c >= (N + 1) * (N + 1)) return RTPN_EINVAL;
    int L = 0;
    while ((L + 1) * (L + 1) <= c) ++L;
    const int mm = c - L * L - L;
    const int M = mm < 0 ? -mm : mm;
    const int t = mm < 0 ? 1 : 0;
    const int sgnM = (M % 2 == 0) ? 1 : -1;
    const int px = t == 0 ? sgnM : -sgnM, py = t == 0 ? 1 : -1, pz = ((L + M) % 2 == 0) ? 1 : -1;
    if (l) *l = L;
    if (m) *m = mm;
    if (slots) {
        slots[0] = px == 1 ? 1 : 2;
        slots[1] = py == 1 ? 1 : 2;
        slots[2] = pz == 1 ? 1 : 2;
    }
    if (cls) *cls = L % 2;
    return RTPN_OK;
}

int rtpn_coupling_dense(int N, int axis, double* out) {
    if (N < 0 || N > 63 || axis < 0 || axis > 2 || !out) return RTPN_EINVAL;
    Model md = build_model(N);
    const size_t n = md.nc;
    std::memset(out, 0, n * n * sizeof(double));
    for (const auto& e : md.nz)
        if (e.axis == axis) out[(size_t)e.a * n + e.b] = e.v;
    return RTPN_OK;
}

int rtpn_create(rtpn_ctx** out, int N, int nx, int ny, int nz, double h, int bc, int precision,
                double dt) {
    if (!out) return fail(nullptr, RTPN_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 0 || N > 63) return fail(nullptr, RTPN_EINVAL, "N must be in 0..63");
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, RTPN_EINVAL, "grid dims must be >= 1");
    if (!(h > 0.0) || !std::isfinite(h)) return fail(nullptr, RTPN_EINVAL, "h must be > 0");
    if (bc != RTPN_BC_PERIODIC && bc != RTPN_BC_VACUUM)
        return fail(nullptr, RTPN_EINVAL, "unknown boundary");
    if (precision != RTPN_FP64 && precision != RTPN_FP32 && precision != RTPN_BF16)
        return fail(nullptr, RTPN_EINVAL, "unknown precision");
    if (dt <= 0.0) dt = 0.3 * h;
    if (!(dt < h / 3.0)) return fail(nullptr, RTPN_ECFL, "dt must be below h/3 (Section 2.1)");
    const long long V = (long long)nx * ny * nz;
    if (V > (1ll << 40)) return fail(nullptr, RTPN_EINVAL, "grid too large");

    rtpn_ctx* ctx = new rtpn_ctx();
    ctx->md = build_model(N);
    ctx->N = N;
    ctx->g = Geom{nx, ny, nz, V, bc, h, h, h};
    ctx->prec = precision;
    ctx->dt = dt;
    ctx->elem = precision == RTPN_FP64 ? 8 : (precision == RTPN_FP32 ? 4 : 2);
    const size_t fac_elem = precision == RTPN_FP64 ? 8 : 4;
    auto bail = [&](int rc) {
        g_create_err = ctx->err;
        release(ctx);
        delete ctx;
        return rc;
    };
    int rc;
    if (cudaStreamCreateWithFlags(&ctx->own, cudaStreamDefault) != cudaSuccess)
        return bail(fail(ctx, RTPN_ECUDA, "stream create failed"));
    ctx->stream = ctx->own;
    cudaError_t e = cudaMalloc(&ctx->u, (size_t)ctx->md.nc * V * ctx->elem);
    if (e != cudaSuccess) return bail(fail(ctx, RTPN_ENOMEM, "state allocation failed"));
    ctx->u_home = ctx->u;
    e = cudaMalloc(&ctx->fac, (size_t)FAC_PLANES * V * fac_elem);
    if (e != cudaSuccess) return bail(fail(ctx, RTPN_ENOMEM, "factor allocation failed"));
    e = cudaMalloc(&ctx->staging, (size_t)V * 8);
    if (e != cudaSuccess) return bail(fail(ctx, RTPN_ENOMEM, "staging allocation failed"));
    e = cudaMalloc(&ctx->partial, (SUM_BLOCKS + 1) * sizeof(double));
    if (e != cudaSuccess) return bail(fail(ctx, RTPN_ENOMEM, "scratch allocation failed"));
    e = cudaMalloc(&ctx->counter, sizeof(unsigned long long));
    if (e != cudaSuccess) return bail(fail(ctx, RTPN_ENOMEM, "scratch allocation failed"));
    e = cudaMalloc(&ctx->status, 8 * sizeof(unsigned));
    if (e != cudaSuccess) return bail(fail(ctx, RTPN_ENOMEM, "status allocation failed"));
    e = cudaMemsetAsync(ctx->status, 0, 8 * sizeof(unsigned), ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, RTPN_ECUDA, cudaGetErrorString(e)));
    if ((rc = upload_tables(ctx))) return bail(rc);
    e = cudaMemsetAsync(ctx->u, 0, (size_t)ctx->md.nc * V * ctx->elem, ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, RTPN_ECUDA, cudaGetErrorString(e)));
    if ((rc = choose_kernel(ctx))) return bail(rc);
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(fail(ctx, RTPN_ECUDA, cudaGetErrorString(e)));
    *out = ctx;
    return RTPN_OK;
}

int rtpn_destroy(rtpn_ctx* ctx) {
    if (!ctx) return RTPN_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    release(ctx);
    delete ctx;
    return RTPN_OK;
}

int rtpn_set_spacing(rtpn_ctx* ctx, double hx, double hy, double hz) {
    if (!ctx) return RTPN_EINVAL;
    if (!(hx > 0.0 && hy > 0.0 && hz > 0.0) || !std::isfinite(hx) || !std::isfinite(hy) ||
        !std::isfinite(hz))
        return fail(ctx, RTPN_EINVAL, "cell sizes must be positive and finite");
    if (!(ctx->dt < std::min(hx, std::min(hy, hz)) / 3.0))
        return fail(ctx, RTPN_ECFL, "dt must be below min(hx, hy, hz)/3 (Section 2.1)");
    const bool cubic = hx == hy && hy == hz;
    // a batch keeps each instance's 1/h in its launch items, built at creation
    if (ctx->batch_member)
        return fail(ctx, RTPN_EUNSUPPORTED, "the spacing of a batch instance is fixed at creation");
    const Geom old = ctx->g;
    ctx->g.h = hx;
    ctx->g.hy = hy;
    ctx->g.hz = hz;
    auto restore = [&](int code, const std::string& msg) {
        ctx->g = old;
        return fail(ctx, code, msg);
    };
    if (!cubic && (ctx->kernel == RTPN_KERNEL_FUSED ||
                   (ctx->kernel == RTPN_KERNEL_WINDOW && !window_extended(ctx->N))))
        return restore(RTPN_EUNSUPPORTED, "the fused kernel, and the window kernel above N = 15, take cubic cells only");
    // the partner tables and the staged kernel's constants carry the spacing: rebuild them
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->table_mem) cudaFree(ctx->table_mem);
    ctx->table_mem = nullptr;
    int rc = upload_tables(ctx);
    if (rc) return rc;
    if (ctx->stage_mem) cudaFree(ctx->stage_mem);
    ctx->stage_mem = nullptr;
    drop_graphs(ctx);
    return choose_kernel(ctx);
}

int rtpn_set_scattering(rtpn_ctx* ctx, const double* f, int count) {
    if (!ctx) return RTPN_EINVAL;
    const bool iso = f == nullptr || count == 0;
    if (!iso) {
        if (count != ctx->N + 1) return fail(ctx, RTPN_EINVAL, "give f_0 .. f_N (count = N + 1)");
        if (f[0] != 1.0) return fail(ctx, RTPN_EINVAL, "f_0 must be 1 (Sigma_s0 = sigma_s)");
        for (int l = 1; l <= ctx->N; ++l)
            if (!(f[l] >= -1.0 && f[l] <= 1.0)) return fail(ctx, RTPN_EINVAL, "f_l must lie in [-1, 1]");
        if (ctx->batch_member)
            return fail(ctx, RTPN_EUNSUPPORTED, "batch instances take isotropic scattering only");
        const bool win_aniso = window_supported(ctx->N, ctx->prec) && window_extended(ctx->N);
        if (ctx->kernel != RTPN_KERNEL_AUTO && ctx->kernel != RTPN_KERNEL_GENERIC &&
            !(ctx->kernel == RTPN_KERNEL_WINDOW && win_aniso))
            return fail(ctx, RTPN_EUNSUPPORTED,
                        "anisotropic scattering runs on the generic kernel and the window kernel up to N = 15");
    }
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    const long long V = ctx->g.V;
    const size_t fac_elem = ctx->prec == RTPN_FP64 ? 8 : 4;
    const int planes = iso ? FAC_PLANES : aniso_planes(ctx->N);
    // new buffers first, so that a failed allocation leaves the context as it was
    double* scat = nullptr;
    void* fac = nullptr;
    if (!iso) {
        cudaError_t e = cudaMalloc(&scat, sizeof(double) * (ctx->N + 1));
        if (e == cudaSuccess) e = cudaMemcpy(scat, f, sizeof(double) * (ctx->N + 1), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (scat) cudaFree(scat);
            cudaGetLastError();
            return fail(ctx, RTPN_ENOMEM, "scattering moments");
        }
    }
    if (planes != ctx->fac_planes) {
        cudaError_t e = cudaMalloc(&fac, (size_t)planes * V * fac_elem);
        if (e != cudaSuccess) {
            if (scat) cudaFree(scat);
            cudaGetLastError();
            return fail(ctx, RTPN_ENOMEM, "factor planes of anisotropic scattering");
        }
    }
    if (ctx->scat) cudaFree(ctx->scat);
    ctx->scat = scat;
    if (fac) {
        cudaFree(ctx->fac);
        ctx->fac = fac;
        ctx->fac_planes = planes;
    }
    drop_graphs(ctx);
    if (ctx->table_mem) cudaFree(ctx->table_mem);
    ctx->table_mem = nullptr;
    int rc = upload_tables(ctx);
    if (!rc) rc = choose_kernel(ctx);
    if (!rc && ctx->media_set) {  // the factors of the media already set, with the new moments
        const double* m = ctx->media;
        if (ctx->prec == RTPN_FP64)
            launch_media_factors<double>(m, m + V, m + 2 * V, (double*)ctx->fac, ctx->g, ctx->dt,
                                         ctx->scat, ctx->N, ctx->stream);
        else
            launch_media_factors<float>(m, m + V, m + 2 * V, (float*)ctx->fac, ctx->g, ctx->dt,
                                        ctx->scat, ctx->N, ctx->stream);
        CUDA_TRY(ctx, cudaGetLastError());
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return rc;
}

int rtpn_set_stream(rtpn_ctx* ctx, void* stream) {
    if (!ctx) return RTPN_EINVAL;
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own;
    return RTPN_OK;
}

int rtpn_set_kernel(rtpn_ctx* ctx, int kernel, int tile_x, int tile_y, int tile_z) {
    return rtpn_set_kernel_ex(ctx, kernel, tile_x, tile_y, tile_z, 0);
}

int rtpn_set_kernel_ex(rtpn_ctx* ctx, int kernel, int tile_x, int tile_y, int tile_z, int depth) {
    if (!ctx) return RTPN_EINVAL;
    if (depth < 0 || depth > 8) return fail(ctx, RTPN_EINVAL, "bad stage depth");
    if (kernel < RTPN_KERNEL_AUTO || kernel > RTPN_KERNEL_FUSED)
        return fail(ctx, RTPN_EINVAL, "unknown kernel");
    if (tile_x < 0 || tile_y < 0 || tile_z < 0) return fail(ctx, RTPN_EINVAL, "bad tile");
    if (kernel == RTPN_KERNEL_FUSED) {
        if ((tile_x && tile_x != 32) || (tile_y && tile_y != 8))
            return fail(ctx, RTPN_EINVAL, "the fused kernel's tile is 32 x 8 cells");
    } else if (kernel != RTPN_KERNEL_STAGE && (tile_x || tile_y || tile_z)) {
        const long long th = (long long)(tile_x ? tile_x : 32) * (tile_y ? tile_y : 4) *
                             (tile_z ? tile_z : 2);
        if (th > 256 || th % 32 != 0)
            return fail(ctx, RTPN_EINVAL, "tile must hold a multiple of 32 threads, at most 256");
    }
    const int old = ctx->kernel, ox = ctx->tx, oy = ctx->ty, oz = ctx->tz, oc = ctx->depth;
    const bool ofs = ctx->tile_from_stage;
    ctx->kernel = kernel;
    drop_graphs(ctx);
    ctx->tx = tile_x;
    ctx->ty = tile_y;
    ctx->tz = tile_z;
    ctx->tile_from_stage = false;
    ctx->depth = kernel == RTPN_KERNEL_STAGE || kernel == RTPN_KERNEL_AUTO ? depth : 0;
    int rc = choose_kernel(ctx);
    if (rc) {
        const std::string msg = ctx->err;
        ctx->kernel = old;
        ctx->tx = ox;
        ctx->ty = oy;
        ctx->tz = oz;
        ctx->depth = oc;
        ctx->tile_from_stage = ofs;
        choose_kernel(ctx);
        ctx->err = msg;
    }
    return rc;
}

int rtpn_set_media(rtpn_ctx* ctx, const void* sigma_a, const void* sigma_s, const void* q,
                   int dtype, int where) {
    if (!ctx || !sigma_a || !sigma_s || !q) return RTPN_EINVAL;
    if (!valid_dtype(dtype) || !valid_where(where)) return fail(ctx, RTPN_EINVAL, "bad dtype/where");
    const long long V = ctx->g.V;
    // the FP64 media stay on the device (the adjoint needs them again)
    if (!ctx->media) CUDA_TRY(ctx, cudaMalloc(&ctx->media, (size_t)3 * V * sizeof(double)));
    double* m = ctx->media;
    const void* srcs[3] = {sigma_a, sigma_s, q};
    const size_t bytes = (size_t)V * dtype_size(dtype);
    int rc = RTPN_OK;
    for (int i = 0; i < 3 && !rc; ++i) {
        double* dst = m + (size_t)i * V;
        const void* src = srcs[i];
        cudaError_t e = cudaSuccess;
        if (dtype == RTPN_DTYPE_F64) {
            e = cudaMemcpyAsync(dst, src, bytes,
                                where == RTPN_HOST ? cudaMemcpyHostToDevice
                                                   : cudaMemcpyDeviceToDevice,
                                ctx->stream);
        } else {
            if (where == RTPN_HOST) {
                e = cudaMemcpyAsync(ctx->staging, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
                src = ctx->staging;
            }
            if (e == cudaSuccess) launch_convert<float, double>((const float*)src, dst, V, ctx->stream);
        }
        if (e != cudaSuccess) rc = fail(ctx, RTPN_ECUDA, cudaGetErrorString(e));
    }
    if (!rc) {
        if (ctx->prec == RTPN_FP64)
            launch_media_factors<double>(m, m + V, m + 2 * V, (double*)ctx->fac, ctx->g, ctx->dt,
                                         ctx->scat, ctx->N, ctx->stream);
        else
            launch_media_factors<float>(m, m + V, m + 2 * V, (float*)ctx->fac, ctx->g, ctx->dt,
                                        ctx->scat, ctx->N, ctx->stream);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = fail(ctx, RTPN_ECUDA, cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(ctx, RTPN_ECUDA, cudaGetErrorString(e));
    ctx->media_set = true;
    return RTPN_OK;
}

int rtpn_set_component(rtpn_ctx* ctx, int c, const void* field, int dtype, int where) {
    if (!ctx || !field) return RTPN_EINVAL;
    if (c < 0 || c >= ctx->md.nc) return fail(ctx, RTPN_EINVAL, "component out of range");
    if (!valid_dtype(dtype) || !valid_where(where)) return fail(ctx, RTPN_EINVAL, "bad dtype/where");
    int rc = put_component(ctx, c, field, dtype, where);
    if (rc) return rc;
    ctx->steps_done = 0;
    if (where == RTPN_HOST) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return RTPN_OK;
}

int rtpn_get_component(rtpn_ctx* ctx, int c, void* field, int dtype, int where) {
    if (!ctx || !field) return RTPN_EINVAL;
    if (c < 0 || c >= ctx->md.nc) return fail(ctx, RTPN_EINVAL, "component out of range");
    if (!valid_dtype(dtype) || !valid_where(where)) return fail(ctx, RTPN_EINVAL, "bad dtype/where");
    int rc = take_component(ctx, c, field, dtype, where);
    if (rc) return rc;
    if (where == RTPN_HOST) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return RTPN_OK;
}

int rtpn_set_moments(rtpn_ctx* ctx, const void* u, int dtype, int where) {
    if (!ctx || !u) return RTPN_EINVAL;
    if (!valid_dtype(dtype) || !valid_where(where)) return fail(ctx, RTPN_EINVAL, "bad dtype/where");
    const size_t plane = (size_t)ctx->g.V * dtype_size(dtype);
    for (int c = 0; c < ctx->md.nc; ++c) {
        int rc = put_component(ctx, c, (const char*)u + (size_t)c * plane, dtype, where);
        if (rc) return rc;
    }
    ctx->steps_done = 0;
    if (where == RTPN_HOST) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return RTPN_OK;
}

int rtpn_get_moments(rtpn_ctx* ctx, void* u, int dtype, int where) {
    if (!ctx || !u) return RTPN_EINVAL;
    if (!valid_dtype(dtype) || !valid_where(where)) return fail(ctx, RTPN_EINVAL, "bad dtype/where");
    const size_t plane = (size_t)ctx->g.V * dtype_size(dtype);
    for (int c = 0; c < ctx->md.nc; ++c) {
        int rc = take_component(ctx, c, (char*)u + (size_t)c * plane, dtype, where);
        if (rc) return rc;
    }
    if (where == RTPN_HOST) CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return RTPN_OK;
}

int rtpn_zero_moments(rtpn_ctx* ctx) {
    if (!ctx) return RTPN_EINVAL;
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->u, 0, (size_t)ctx->md.nc * ctx->g.V * ctx->elem, ctx->stream));
    ctx->steps_done = 0;
    return RTPN_OK;
}

int rtpn_step(rtpn_ctx* ctx, int k) {
    if (!ctx || k < 0) return RTPN_EINVAL;
    if (!ctx->media_set) return fail(ctx, RTPN_ESTATE, "rtpn_set_media has not been called");
    if (k == 0) return RTPN_OK;
    bool fused = ctx->active_kernel == RTPN_KERNEL_FUSED;
    if (fused) {
        // a caller's capture keeps the pointers it saw: the two-pass schedule stays in one buffer
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CUDA_TRY(ctx, cudaStreamIsCapturing(ctx->stream, &cap));
        fused = cap == cudaStreamCaptureStatusNone;
    }
    int rc = run_pass(ctx, 1, FAC_HALF, ctx->stream);
    if (!rc) rc = launch_pairs(ctx, k - 1, fused);
    if (fused) {
        if (!rc) rc = fused_pass(ctx, ctx->u, ctx->u_alt, FAC_HALF, ctx->stream);
        if (!rc) std::swap(ctx->u, ctx->u_alt);
    } else {
        if (!rc) rc = run_pass(ctx, 0, FAC_FULL, ctx->stream);
        if (!rc) rc = run_pass(ctx, 1, FAC_HALF, ctx->stream);
    }
    if (!rc) ctx->steps_done += k;
    return rc;
}

int rtpn_substep(rtpn_ctx* ctx, int cls, int half) {
    if (!ctx || cls < 0 || cls > 1 || half < 0 || half > 1) return RTPN_EINVAL;
    if (cls == 0 && half) return fail(ctx, RTPN_EINVAL, "the even class has no half-step factors");
    if (!ctx->media_set) return fail(ctx, RTPN_ESTATE, "rtpn_set_media has not been called");
    return run_pass(ctx, cls, half ? FAC_HALF : FAC_FULL, ctx->stream);
}

int rtpn_copy_planes(rtpn_ctx* dst, int dst_z, rtpn_ctx* src, int src_z, int nz, int cls) {
    if (!dst || !src || nz < 0 || cls < -1 || cls > 1) return RTPN_EINVAL;
    if (src->N != dst->N || src->prec != dst->prec || src->g.nx != dst->g.nx || src->g.ny != dst->g.ny)
        return fail(dst, RTPN_EINVAL, "copy_planes: the contexts differ in order, precision, nx or ny");
    if (src_z < 0 || dst_z < 0 || src_z + nz > src->g.nz || dst_z + nz > dst->g.nz)
        return fail(dst, RTPN_EINVAL, "copy_planes: planes outside a grid");
    if (src == dst && nz > 0 && src_z < dst_z + nz && dst_z < src_z + nz)
        return fail(dst, RTPN_EINVAL, "copy_planes: overlapping planes of one context");
    if (nz == 0) return RTPN_OK;
    // the components of a class are contiguous in the internal order (class 0 first)
    const int c0 = cls == 1 ? dst->md.ne : 0;
    const int n = cls == -1 ? dst->md.nc : (cls == 0 ? dst->md.ne : dst->md.no);
    const size_t plane = (size_t)dst->g.nx * dst->g.ny * dst->elem;
    const char* sp = (const char*)src->u + ((size_t)c0 * src->g.V + (size_t)src_z * dst->g.nx * dst->g.ny) * dst->elem;
    char* dp = (char*)dst->u + ((size_t)c0 * dst->g.V + (size_t)dst_z * dst->g.nx * dst->g.ny) * dst->elem;
    // the copy runs on dst's stream after src's queued work, and src's later work runs after it
    cudaEvent_t ev = nullptr;
    if (src->stream != dst->stream) {
        CUDA_TRY(dst, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CUDA_TRY(dst, cudaEventRecord(ev, src->stream));
        CUDA_TRY(dst, cudaStreamWaitEvent(dst->stream, ev, 0));
    }
    cudaError_t e = cudaMemcpy2DAsync(dp, (size_t)dst->g.V * dst->elem, sp, (size_t)src->g.V * dst->elem,
                                      (size_t)nz * plane, (size_t)n, cudaMemcpyDeviceToDevice, dst->stream);
    if (ev) {
        if (e == cudaSuccess) e = cudaEventRecord(ev, dst->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(src->stream, ev, 0);
        cudaEventDestroy(ev);
    }
    if (e != cudaSuccess) return fail(dst, RTPN_ECUDA, std::string("copy_planes: ") + cudaGetErrorString(e));
    return RTPN_OK;
}

int rtpn_sum_u0(rtpn_ctx* ctx, double* out) {
    if (!ctx || !out) return RTPN_EINVAL;
    const void* u0 = comp_ptr(ctx, ctx->md.internal_of_abi[0]);
    with_storage(ctx->prec, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        launch_sum<S>((const S*)u0, ctx->g.V, ctx->partial, SUM_BLOCKS, ctx->partial + SUM_BLOCKS,
                      ctx->stream);
    });
    CHECK_LAUNCH(ctx);
    CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->partial + SUM_BLOCKS, sizeof(double),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return RTPN_OK;
}

int rtpn_count_nonfinite(rtpn_ctx* ctx, long long* out) {
    if (!ctx || !out) return RTPN_EINVAL;
    with_storage(ctx->prec, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        launch_count_nonfinite<S>((const S*)ctx->u, (long long)ctx->md.nc * ctx->g.V, ctx->counter,
                                  ctx->stream);
    });
    CHECK_LAUNCH(ctx);
    unsigned long long c = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&c, ctx->counter, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    *out = (long long)c;
    return c ? fail(ctx, RTPN_ENONFINITE, "non-finite values in the state") : RTPN_OK;
}

int rtpn_synchronize(rtpn_ctx* ctx) {
    if (!ctx) return RTPN_EINVAL;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    unsigned st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    CUDA_TRY(ctx, cudaMemcpy(st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st[0]) {
        std::string rec;
        for (int i = 0; i < 8; ++i) rec += (i ? " " : "") + std::to_string(st[i]);
        CUDA_TRY(ctx, cudaMemset(ctx->status, 0, sizeof(st)));
        if (st[0] & 1u)
            return fail(ctx, RTPN_ETIMEOUT, "a bounded wait in a staged kernel ran out [" + rec + "]");
        return fail(ctx, RTPN_ECUDA, "a staged-kernel self-check failed [" + rec + "]");
    }
    CUDA_TRY(ctx, cudaMemset(ctx->status, 0, sizeof(st)));
    return RTPN_OK;
}

int rtpn_test_wait_timeout(rtpn_ctx* ctx, int cls, long long wait_limit) {
    if (!ctx || cls < 0 || cls > 1 || wait_limit < 1) return RTPN_EINVAL;
    if (ctx->active_kernel != RTPN_KERNEL_STAGE)
        return fail(ctx, RTPN_EUNSUPPORTED, "the staged kernel is not active");
    if (!ctx->media_set) return fail(ctx, RTPN_ESTATE, "rtpn_set_media has not been called");
    // stage 1 of every CTA's sequence is never issued
    int rc = launch_stage(ctx, cls, FAC_FULL, ctx->stream, 1, wait_limit);
    if (rc) return fail(ctx, RTPN_ECUDA, cudaGetErrorString((cudaError_t)rc));
    return RTPN_OK;
}

int rtpn_get_info(const rtpn_ctx* ctx, rtpn_info* out) {
    if (!ctx || !out) return RTPN_EINVAL;
    out->N = ctx->N;
    out->n_c = ctx->md.nc;
    out->n_even = ctx->md.ne;
    out->n_odd = ctx->md.no;
    out->nx = ctx->g.nx;
    out->ny = ctx->g.ny;
    out->nz = ctx->g.nz;
    out->bc = ctx->g.bc;
    out->precision = ctx->prec;
    out->kernel = ctx->active_kernel;
    out->h = ctx->g.h;
    out->hy = ctx->g.hy;
    out->hz = ctx->g.hz;
    out->dt = ctx->dt;
    out->state_bytes = (size_t)ctx->md.nc * ctx->g.V * ctx->elem;
    out->factor_bytes = (size_t)ctx->fac_planes * ctx->g.V * (ctx->prec == RTPN_FP64 ? 8 : 4);
    out->steps_done = ctx->steps_done;
    out->tile[0] = ctx->tx;
    out->tile[1] = ctx->ty;
    out->tile[2] = ctx->tz;
    out->depth = ctx->active_kernel == RTPN_KERNEL_STAGE ? ctx->depth : 1;
    return RTPN_OK;
}

const char* rtpn_last_error(const rtpn_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

}  // extern "C"
