// Batched form: many independent P_N instances of uneven order and size advanced together.
//
// Each pass of the merged Strang schedule (Eq. 6) is one persistent launch per order present in the
// batch (heaviest order first), each over the tiles of every instance of that order: CTAs take
// tiles from the order's work counter (largest instances first) and run the same compile-time
// register-window cell body as the single-instance kernel.  One launch per order rather than one
// for all orders: a kernel that dispatches on N at run time is compiled for the registers of its
// largest order, which caps the occupancy of every smaller order's tiles.  Instances are
// independent, so a pass has no cross-instance dependence; consecutive passes are ordered by the
// stream.  Whole k-step sequences are replayed from captured CUDA graphs.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "window_impl.cuh"

#define RTPN_BATCH_ORDERS(X) X(1) X(3) X(5) X(7) X(9) X(15)

namespace rtpn {
namespace bat {

using win::Args;

#define RTPN_BCONST(n)                                                                   \
    static __constant__ float c_coef_##n##_0[win::class_size(n, 1) * 10];               \
    static __constant__ float c_coef_##n##_1[win::class_size(n, 0) * 10];
RTPN_BATCH_ORDERS(RTPN_BCONST)
#undef RTPN_BCONST

struct Inst {
    void* u;
    const float* fac;
    long long V;
    long long block0;  // first work item of this instance
    int nx, ny, nz, bc;
    float inv_h;
    int ntx, nty, ntz;
};

template <int N, int A>
__device__ __forceinline__ const float* coef_of() {
#define RTPN_CASE(n) \
    if constexpr (N == n) return A == 0 ? c_coef_##n##_0 : c_coef_##n##_1;
    RTPN_BATCH_ORDERS(RTPN_CASE)
#undef RTPN_CASE
    return nullptr;
}

// Persistent, for the instances of one order N: each CTA repeatedly takes the next tile index from
// *counter until all of the group's tiles are done.
template <int N, int A, typename S>
__global__ void __launch_bounds__(256) k_batch(const Inst* __restrict__ inst, int count,
                                               long long items, int tx, int ty, int tz,
                                               int fac_ofs, unsigned long long* counter) {
    __shared__ long long s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long it = s_item;
        __syncthreads();
        if (it >= items) break;
        int lo = 0, hi = count - 1;  // last instance with block0 <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (inst[mid].block0 <= it) lo = mid; else hi = mid - 1;
        }
        const Inst& I = inst[lo];
        Args a;
        a.u = I.u;
        a.fac = I.fac;
        a.V = I.V;
        a.nx = I.nx;
        a.ny = I.ny;
        a.nz = I.nz;
        a.bc = I.bc;
        a.fac_ofs = fac_ofs;
        a.inv_h = I.inv_h;
        a.tx = tx;
        a.ty = ty;
        a.tz = tz;
        a.ntx = I.ntx;
        a.nty = I.nty;
        a.ntz = I.ntz;
        int x, y, z;
        if (win::cell_of(a, (int)(it - I.block0), threadIdx.x, &x, &y, &z))
            win::substep_cell<N, A, S>(a, coef_of<N, A>(), x, y, z);
    }
}

bool supported(int N) {
    switch (N) {
#define RTPN_SUP(n) case n:
        RTPN_BATCH_ORDERS(RTPN_SUP)
#undef RTPN_SUP
        return true;
        default:
            return false;
    }
}

int upload_constants(const Model& md) {
    static std::mutex mu;
    static std::set<std::pair<int, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({md.N, dev})) return 0;
    for (int A = 0; A < 2; ++A) {
        std::vector<float> t;
        if (!win::coef_table(md, A, &t)) return (int)cudaErrorInvalidValue;
        const void* sym = nullptr;
        switch (md.N) {
#define RTPN_SYM(n) \
    case n: sym = A == 0 ? (const void*)&c_coef_##n##_0 : (const void*)&c_coef_##n##_1; break;
            RTPN_BATCH_ORDERS(RTPN_SYM)
#undef RTPN_SYM
            default:
                return (int)cudaErrorNotSupported;
        }
        e = cudaMemcpyToSymbol(sym, t.data(), t.size() * sizeof(float));
        if (e != cudaSuccess) return (int)e;
    }
    done.insert({md.N, dev});
    return 0;
}

}  // namespace bat
}  // namespace rtpn

using namespace rtpn;

// the instances of one order: descriptors [first, first + count) of the device array, tiles
// numbered from 0 within the group, one persistent launch of `grid` CTAs per pass
struct BatchGroup {
    int N = 0, first = 0, count = 0, grid = 0;
    long long items = 0;
};

struct rtpn_batch {
    std::vector<rtpn_ctx*> ctx;         // one context per instance (memory, media, moments)
    std::vector<int> order;             // instances sorted heaviest first (order, then cells)
    std::vector<BatchGroup> groups;     // one per order present, heaviest order first
    bat::Inst* d_inst = nullptr;        // device descriptors
    unsigned long long* counter = nullptr;  // one work counter per group
    int prec = RTPN_FP32;
    int tx = 32, ty = 4, tz = 2;
    cudaStream_t stream = nullptr, own = nullptr;
    std::map<int, cudaGraphExec_t> graphs;
    bool media_set_all = false;
    std::string err;
};

namespace {

int bfail(rtpn_batch* b, int code, const std::string& msg) {
    if (b) b->err = msg;
    return code;
}

void drop_graphs(rtpn_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// the kernel of order N, class A, storage S (for the occupancy query)
template <int A, typename S>
const void* kernel_of(int N) {
    switch (N) {
#define RTPN_KER(n) \
    case n:         \
        return (const void*)bat::k_batch<n, A, S>;
        RTPN_BATCH_ORDERS(RTPN_KER)
#undef RTPN_KER
        default:
            return nullptr;
    }
}

// (re)build the device descriptors and the order groups for the current tile
int build_items(rtpn_batch* b) {
    std::vector<bat::Inst> h;
    b->groups.clear();
    for (int idx : b->order) {
        rtpn_ctx* c = b->ctx[idx];
        if (b->groups.empty() || b->groups.back().N != c->N) {
            BatchGroup gr;
            gr.N = c->N;
            gr.first = (int)h.size();
            b->groups.push_back(gr);
        }
        BatchGroup& gr = b->groups.back();
        bat::Inst I{};
        I.u = c->u;
        I.fac = (const float*)c->fac;
        I.V = c->g.V;
        I.nx = c->g.nx;
        I.ny = c->g.ny;
        I.nz = c->g.nz;
        I.bc = c->g.bc;
        I.inv_h = (float)(1.0 / c->g.h);
        I.ntx = (I.nx + b->tx - 1) / b->tx;
        I.nty = (I.ny + b->ty - 1) / b->ty;
        I.ntz = (I.nz + b->tz - 1) / b->tz;
        I.block0 = gr.items;
        gr.items += (long long)I.ntx * I.nty * I.ntz;
        ++gr.count;
        h.push_back(I);
    }
    cudaError_t e = cudaMemcpy(b->d_inst, h.data(), h.size() * sizeof(bat::Inst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(b, RTPN_ECUDA, cudaGetErrorString(e));
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = b->tx * b->ty * b->tz;
    for (auto& gr : b->groups) {
        // the two classes' kernels differ little in registers: size the grid by the even one's
        const void* k = b->prec == RTPN_BF16 ? kernel_of<0, __nv_bfloat16>(gr.N) : kernel_of<0, float>(gr.N);
        int per_sm = 0;
        e = k ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0) : cudaErrorInvalidValue;
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        gr.grid = (int)std::max(1ll, std::min((long long)sms * per_sm, gr.items));
    }
    drop_graphs(b);
    return RTPN_OK;
}

template <int A, typename S>
void launch_group(const BatchGroup& gr, rtpn_batch* b, int fac_ofs, unsigned long long* counter, cudaStream_t st) {
    const int threads = b->tx * b->ty * b->tz;
    switch (gr.N) {
#define RTPN_LAUNCH(n)                                                                              \
    case n:                                                                                         \
        bat::k_batch<n, A, S><<<gr.grid, threads, 0, st>>>(b->d_inst + gr.first, gr.count, gr.items, \
                                                           b->tx, b->ty, b->tz, fac_ofs, counter);  \
        break;
        RTPN_BATCH_ORDERS(RTPN_LAUNCH)
#undef RTPN_LAUNCH
        default:
            break;
    }
}

int batch_pass(rtpn_batch* b, int cls, int fac_ofs, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b->counter, 0, b->groups.size() * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return bfail(b, RTPN_ECUDA, cudaGetErrorString(e));
    for (size_t k = 0; k < b->groups.size(); ++k) {
        const BatchGroup& gr = b->groups[k];
        unsigned long long* ctr = b->counter + k;
        if (b->prec == RTPN_BF16) {
            if (cls == 0) launch_group<0, __nv_bfloat16>(gr, b, fac_ofs, ctr, st);
            else launch_group<1, __nv_bfloat16>(gr, b, fac_ofs, ctr, st);
        } else {
            if (cls == 0) launch_group<0, float>(gr, b, fac_ofs, ctr, st);
            else launch_group<1, float>(gr, b, fac_ofs, ctr, st);
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, RTPN_ECUDA, std::string("batch kernel: ") + cudaGetErrorString(e));
    return RTPN_OK;
}

int batch_pairs(rtpn_batch* b, int pairs, cudaStream_t st) {
    for (int p = 0; p < pairs; ++p) {
        int rc = batch_pass(b, 0, FAC_FULL, st);
        if (!rc) rc = batch_pass(b, 1, FAC_FULL, st);
        if (rc) return rc;
    }
    return RTPN_OK;
}

int launch_pairs(rtpn_batch* b, int pairs) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(b->stream, &cap);
    if (e != cudaSuccess) return bfail(b, RTPN_ECUDA, cudaGetErrorString(e));
    if (cap != cudaStreamCaptureStatusNone) return batch_pairs(b, pairs, b->stream);
    for (int s : {64, 8, 1}) {
        while (pairs >= s) {
            auto it = b->graphs.find(s);
            if (it == b->graphs.end()) {
                cudaGraph_t g = nullptr;
                e = cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) return bfail(b, RTPN_ECUDA, cudaGetErrorString(e));
                int rc = batch_pairs(b, s, b->own);
                e = cudaStreamEndCapture(b->own, &g);
                if (rc) {
                    if (g) cudaGraphDestroy(g);
                    return rc;
                }
                if (e != cudaSuccess) return bfail(b, RTPN_ECUDA, cudaGetErrorString(e));
                cudaGraphExec_t x = nullptr;
                e = cudaGraphInstantiate(&x, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return bfail(b, RTPN_ECUDA, cudaGetErrorString(e));
                it = b->graphs.emplace(s, x).first;
            }
            e = cudaGraphLaunch(it->second, b->stream);
            if (e != cudaSuccess) return bfail(b, RTPN_ECUDA, cudaGetErrorString(e));
            pairs -= s;
        }
    }
    return RTPN_OK;
}

void release(rtpn_batch* b) {
    drop_graphs(b);
    for (auto* c : b->ctx) rtpn_destroy(c);
    b->ctx.clear();
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->counter) cudaFree(b->counter);
    if (b->own) cudaStreamDestroy(b->own);
}

bool valid_index(rtpn_batch* b, int i) { return b && i >= 0 && i < (int)b->ctx.size(); }

}  // namespace

extern "C" {

int rtpn_batch_create(rtpn_batch** out, int count, const int* N, const int* nx, const int* ny,
                      const int* nz, const double* h, const int* bc, const double* dt,
                      int precision) {
    if (!out || count < 1 || !N || !nx || !ny || !nz || !h || !bc) return RTPN_EINVAL;
    *out = nullptr;
    if (precision != RTPN_FP32 && precision != RTPN_BF16) return RTPN_EUNSUPPORTED;
    for (int i = 0; i < count; ++i)
        if (!bat::supported(N[i])) return RTPN_EUNSUPPORTED;
    rtpn_batch* b = new rtpn_batch();
    b->prec = precision;
    for (int i = 0; i < count; ++i) {
        rtpn_ctx* c = nullptr;
        int rc = rtpn_create(&c, N[i], nx[i], ny[i], nz[i], h[i], bc[i], precision, dt ? dt[i] : 0.0);
        if (rc) {
            release(b);
            delete b;
            return rc;
        }
        c->batch_member = true;
        b->ctx.push_back(c);
        rc = bat::upload_constants(c->md);
        if (rc) {
            release(b);
            delete b;
            return RTPN_ECUDA;
        }
    }
    // heaviest instances (largest order, then most cells) take the first work items
    b->order.resize(count);
    for (int i = 0; i < count; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        if (N[x] != N[y]) return N[x] > N[y];
        return (long long)nx[x] * ny[x] * nz[x] > (long long)nx[y] * ny[y] * nz[y];
    });
    if (cudaMalloc(&b->d_inst, sizeof(bat::Inst) * count) != cudaSuccess ||
        cudaMalloc(&b->counter, sizeof(unsigned long long) * count) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->own, cudaStreamDefault) != cudaSuccess) {
        release(b);
        delete b;
        return RTPN_ENOMEM;
    }
    b->stream = b->own;
    for (auto* c : b->ctx) rtpn_set_stream(c, b->own);
    int rc = build_items(b);
    if (rc) {
        release(b);
        delete b;
        return rc;
    }
    *out = b;
    return RTPN_OK;
}

int rtpn_batch_destroy(rtpn_batch* b) {
    if (!b) return RTPN_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    release(b);
    delete b;
    return RTPN_OK;
}

int rtpn_batch_count(const rtpn_batch* b) { return b ? (int)b->ctx.size() : RTPN_EINVAL; }

int rtpn_batch_set_stream(rtpn_batch* b, void* stream) {
    if (!b) return RTPN_EINVAL;
    b->stream = stream ? (cudaStream_t)stream : b->own;
    for (auto* c : b->ctx) rtpn_set_stream(c, b->stream);
    return RTPN_OK;
}

int rtpn_batch_set_tile(rtpn_batch* b, int tx, int ty, int tz) {
    if (!b || tx < 1 || ty < 1 || tz < 1) return RTPN_EINVAL;
    const int th = tx * ty * tz;
    if (th > 256 || th % 32 != 0) return bfail(b, RTPN_EINVAL, "tile threads must be k*32 <= 256");
    cudaStreamSynchronize(b->stream);
    b->tx = tx;
    b->ty = ty;
    b->tz = tz;
    return build_items(b);
}

int rtpn_batch_get_tile(const rtpn_batch* b, int* tx, int* ty, int* tz) {
    if (!b || !tx || !ty || !tz) return RTPN_EINVAL;
    *tx = b->tx;
    *ty = b->ty;
    *tz = b->tz;
    return RTPN_OK;
}

rtpn_ctx* rtpn_batch_instance(rtpn_batch* b, int i) { return valid_index(b, i) ? b->ctx[i] : nullptr; }

int rtpn_batch_step(rtpn_batch* b, int k) {
    if (!b || k < 0) return RTPN_EINVAL;
    for (auto* c : b->ctx)
        if (!c->media_set) return bfail(b, RTPN_ESTATE, "media not set for every instance");
    if (k == 0) return RTPN_OK;
    int rc = batch_pass(b, 1, FAC_HALF, b->stream);
    if (!rc) rc = launch_pairs(b, k - 1);
    if (!rc) rc = batch_pass(b, 0, FAC_FULL, b->stream);
    if (!rc) rc = batch_pass(b, 1, FAC_HALF, b->stream);
    if (!rc)
        for (auto* c : b->ctx) c->steps_done += k;
    return rc;
}

int rtpn_batch_step_looped(rtpn_batch* b, int k) {
    if (!b || k < 0) return RTPN_EINVAL;
    for (auto* c : b->ctx) {
        if (!c->media_set) return bfail(b, RTPN_ESTATE, "media not set for every instance");
        int rc = rtpn_set_kernel(c, RTPN_KERNEL_WINDOW, b->tx, b->ty, b->tz);
        if (rc) return bfail(b, rc, c->err);
    }
    if (k == 0) return RTPN_OK;
    auto all = [&](int cls, int half) {
        for (auto* c : b->ctx) {
            int rc = rtpn_substep(c, cls, half);
            if (rc) return bfail(b, rc, c->err);
        }
        return (int)RTPN_OK;
    };
    int rc = all(1, 1);
    for (int s = 1; s < k && !rc; ++s) {
        rc = all(0, 0);
        if (!rc) rc = all(1, 0);
    }
    if (!rc) rc = all(0, 0);
    if (!rc) rc = all(1, 1);
    if (!rc)
        for (auto* c : b->ctx) c->steps_done += k;
    return rc;
}

int rtpn_batch_synchronize(rtpn_batch* b) {
    if (!b) return RTPN_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? RTPN_OK : bfail(b, RTPN_ECUDA, cudaGetErrorString(e));
}

const char* rtpn_batch_last_error(const rtpn_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
