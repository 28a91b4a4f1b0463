// Dispatch to the compiled fused step kernels (fused.cu, one translation unit per order) and their
// __constant__ coefficient tables.
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "fused_impl.cuh"
#include "fused_variants.h"

namespace rtpn {
namespace fus {

#define RTPN_DECL(n)                                                                   \
    int fused_upload_N_##n(const float*, int, const float*, int);                     \
    int fused_launch_N_##n(int, const Args&, cudaStream_t);
RTPN_FUSED_ORDERS(RTPN_DECL)
#undef RTPN_DECL

struct Variant {
    int N;
    int (*upload)(const float*, int, const float*, int);
    int (*launch)(int, const Args&, cudaStream_t);
};

#define RTPN_ENTRY(n) Variant{n, fused_upload_N_##n, fused_launch_N_##n},
static const Variant kVariants[] = {RTPN_FUSED_ORDERS(RTPN_ENTRY)};
#undef RTPN_ENTRY

static const Variant* find(int N) {
    for (const auto& v : kVariants)
        if (v.N == N) return &v;
    return nullptr;
}

}  // namespace fus

bool fused_supported(int N, int precision) {
    return precision != RTPN_FP64 && fus::find(N) != nullptr;
}

int fused_prepare(const Model& md, int precision) {
    static std::mutex mu;
    static std::set<std::pair<int, int>> done;  // (N, device)
    const fus::Variant* v = fus::find(md.N);
    if (!v || precision == RTPN_FP64) return (int)cudaErrorNotSupported;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({md.N, dev})) return 0;
    std::vector<float> te, to;
    if (!win::coef_table(md, 0, &te) || !win::coef_table(md, 1, &to)) return (int)cudaErrorInvalidValue;
    int rc = v->upload(te.data(), (int)te.size(), to.data(), (int)to.size());
    if (rc) return rc;
    done.insert({md.N, dev});
    return 0;
}

int launch_fused(int N, int precision, const FusedLaunch& f, cudaStream_t st) {
    const fus::Variant* v = fus::find(N);
    if (!v) return (int)cudaErrorNotSupported;
    if (f.x == f.y) return (int)cudaErrorInvalidValue;
    fus::Args a;
    a.x = f.x;
    a.y = f.y;
    a.fac = f.fac;
    a.V = f.g.V;
    a.nx = f.g.nx;
    a.ny = f.g.ny;
    a.nz = f.g.nz;
    a.bc = f.g.bc;
    a.fac_even = FAC_FULL;
    a.fac_odd = f.fac_odd;
    a.inv_h = (float)(1.0 / f.g.h);
    a.zc = f.zc > 0 ? (f.zc < a.nz ? f.zc : a.nz) : 0;
    a.ntx = (a.nx + fus::TX - 1) / fus::TX;
    a.nty = (a.ny + fus::TY - 1) / fus::TY;
    a.nzc = 0;  // set by the variant once zc is known
    return v->launch(precision, a, st);
}

}  // namespace rtpn
