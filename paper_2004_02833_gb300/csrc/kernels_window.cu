// Dispatch to the compiled register-window variants and their __constant__ coefficient tables.
#include <cstdlib>
#include <mutex>
#include <set>
#include <string>
#include <unordered_map>
#include <utility>

#include "window_impl.cuh"
#include "window_variants.h"

namespace rtpn {
namespace win {

#define RTPN_DECL(n)                                                                   \
    int window_upload_N_##n##_0(const float*, int);                                   \
    int window_upload_N_##n##_1(const float*, int);                                   \
    int window_launch_N_##n##_0(int, const Args&, cudaStream_t);                      \
    int window_launch_N_##n##_1(int, const Args&, cudaStream_t);
RTPN_WINDOW_ORDERS(RTPN_DECL)
#undef RTPN_DECL

struct Variant {
    int N;
    int (*upload[2])(const float*, int);
    int (*launch[2])(int, const Args&, cudaStream_t);
};

#define RTPN_ENTRY(n)                                                                  \
    Variant{n,                                                                         \
            {window_upload_N_##n##_0, window_upload_N_##n##_1},                        \
            {window_launch_N_##n##_0, window_launch_N_##n##_1}},
static const Variant kVariants[] = {RTPN_WINDOW_ORDERS(RTPN_ENTRY)};
#undef RTPN_ENTRY

static const Variant* find(int N) {
    for (const auto& v : kVariants)
        if (v.N == N) return &v;
    return nullptr;
}

}  // namespace win

bool window_supported(int N, int precision) {
    return precision != RTPN_FP64 && win::find(N) != nullptr;
}

bool window_extended(int N) { return N <= win::kExtendedMaxN; }

int window_prepare(const Model& md, double, int precision) {
    static std::mutex mu;
    static std::set<std::pair<int, int>> done;  // (N, device)
    const win::Variant* v = win::find(md.N);
    if (!v || precision == RTPN_FP64) return (int)cudaErrorNotSupported;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({md.N, dev})) return 0;
    for (int A = 0; A < 2; ++A) {
        std::vector<float> t;
        if (!win::coef_table(md, A, &t)) return (int)cudaErrorInvalidValue;
        int rc = v->upload[A](t.data(), (int)t.size());
        if (rc) return rc;
    }
    done.insert({md.N, dev});
    return 0;
}

int launch_window(int N, int precision, const WindowLaunch& w, cudaStream_t st) {
    const win::Variant* v = win::find(N);
    if (!v) return (int)cudaErrorNotSupported;
    win::Args a;
    a.u = w.u;
    a.fac = w.fac;
    a.V = w.g.V;
    a.nx = w.g.nx;
    a.ny = w.g.ny;
    a.nz = w.g.nz;
    a.bc = w.g.bc;
    a.fac_ofs = w.fac_ofs;
    a.inv_h = (float)(1.0 / w.g.h);
    a.sy = (float)(w.g.h / w.g.hy);  // exactly 1 for cubic cells
    a.sz = (float)(w.g.h / w.g.hz);
    a.aniso = w.aniso ? 1 : 0;
    a.tx = w.tx > 0 ? w.tx : 32;
    a.ty = w.ty > 0 ? w.ty : 4;
    a.tz = w.tz > 0 ? w.tz : 2;
    if (a.tx * a.ty * a.tz > 256 || (a.tx * a.ty * a.tz) % 32 != 0) return (int)cudaErrorInvalidValue;
    a.ntx = (a.nx + a.tx - 1) / a.tx;
    a.nty = (a.ny + a.ty - 1) / a.ty;
    a.ntz = (a.nz + a.tz - 1) / a.tz;
    return v->launch[w.cls](precision, a, st);
}

}  // namespace rtpn
