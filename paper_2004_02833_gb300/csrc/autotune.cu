// Autotuner for the CTA tile of the register-window kernels (single instance and batched form).
//
// Each candidate tile is timed on the object's own data: the state is copied aside, `reps` pairs of
// (even pass, odd pass) are timed with CUDA events on the object's stream after one warm-up pair,
// and the state is copied back, so tuning leaves the moments unchanged.  Results are cached per
// (order(s), precision, boundary, grid, device) for the life of the process and, if the environment
// variable RTPN_TUNE_CACHE names a file, appended to it and read back by later processes.
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "rtpn_internal.h"

namespace {

struct Tile {
    int x, y, z;
    int c = 0;  // stage buffers (staged kernel), 0 = not applicable
};

const Tile kCandidates[] = {{32, 1, 1},  {32, 2, 1}, {32, 4, 1}, {32, 8, 1}, {32, 1, 2}, {32, 2, 2},
                            {32, 4, 2},  {32, 1, 4}, {32, 2, 4}, {32, 1, 8}, {64, 1, 1}, {64, 2, 1},
                            {64, 1, 2},  {64, 2, 2}, {64, 4, 1}, {16, 2, 4}, {16, 4, 4}, {16, 2, 8},
                            {8, 8, 4},   {8, 4, 8},  {128, 1, 1}, {128, 2, 1}, {128, 1, 2}, {256, 1, 1}};

std::mutex g_mu;
std::map<std::string, std::pair<Tile, double>> g_cache;
bool g_file_loaded = false;

void load_file() {
    if (g_file_loaded) return;
    g_file_loaded = true;
    const char* path = std::getenv("RTPN_TUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        const size_t bar = line.rfind('|');
        if (bar == std::string::npos) continue;
        std::istringstream in(line.substr(bar + 1));
        Tile t;
        double ms;
        if (in >> t.x >> t.y >> t.z >> t.c >> ms) g_cache[line.substr(0, bar)] = {t, ms};
    }
}

void store_file(const std::string& key, Tile t, double ms) {
    const char* path = std::getenv("RTPN_TUNE_CACHE");
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << key << "|" << t.x << " " << t.y << " " << t.z << " " << t.c << " " << ms << "\n";
}

std::string device_key() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "dev?";
    return std::string(p.name);
}

// Times `reps` pass pairs for every candidate via `run_pair(stream)`; `set_tile(t)` applies one.
template <typename SetTile, typename RunPair>
int sweep(cudaStream_t st, int reps, const std::vector<Tile>& cands, SetTile set_tile, RunPair run_pair,
          Tile* best, double* best_ms) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return RTPN_ECUDA;
    *best_ms = -1.0;
    int rc = RTPN_OK;
    for (const Tile& t : cands) {
        if (set_tile(t) != RTPN_OK) continue;  // tile not valid for this object
        if ((rc = run_pair(st))) break;        // warm-up
        cudaEventRecord(a, st);
        for (int r = 0; r < reps && !rc; ++r) rc = run_pair(st);
        cudaEventRecord(b, st);
        if (rc) break;
        if (cudaEventSynchronize(b) != cudaSuccess) {
            rc = RTPN_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double per = ms / reps;
        if (*best_ms < 0 || per < *best_ms) {
            *best_ms = per;
            *best = t;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!rc && *best_ms < 0) rc = RTPN_EUNSUPPORTED;
    return rc;
}

}  // namespace

extern "C" {

int rtpn_autotune(rtpn_ctx* ctx, int reps, int tile[3], double* ms_per_step) {
    if (!ctx || reps < 1) return RTPN_EINVAL;
    if (!ctx->media_set) {
        ctx->err = "rtpn_set_media has not been called";
        return RTPN_ESTATE;
    }
    if (ctx->active_kernel != RTPN_KERNEL_WINDOW && ctx->active_kernel != RTPN_KERNEL_STAGE) {
        ctx->err = "the autotuner tunes the window and staged kernels, neither is active";
        return RTPN_EUNSUPPORTED;
    }
    const int kernel = ctx->active_kernel;
    std::ostringstream k;
    k << "single kernel=" << kernel << " N=" << ctx->N << " prec=" << ctx->prec << " bc=" << ctx->g.bc << " grid="
      << ctx->g.nx << "x" << ctx->g.ny << "x" << ctx->g.nz << " dev=" << device_key();
    const std::string key = k.str();
    Tile best{ctx->tx, ctx->ty, ctx->tz, ctx->depth};
    double best_ms = -1.0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        load_file();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            best = it->second.first;
            best_ms = it->second.second;
        }
    }
    std::vector<Tile> cands;
    if (kernel == RTPN_KERNEL_STAGE) {
        int v[4 * 64];
        const int n = rtpn::stage_variants_of(ctx->N, ctx->prec, v, 64);
        for (int i = 0; i < n; ++i) cands.push_back({v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]});
    } else {
        for (const Tile& t : kCandidates) cands.push_back(t);
    }
    if (best_ms < 0) {
        const size_t bytes = (size_t)ctx->md.nc * ctx->g.V * ctx->elem;
        void* snap = nullptr;
        if (cudaMalloc(&snap, bytes) != cudaSuccess) {
            cudaGetLastError();
            ctx->err = "no device memory for the state snapshot the tuner needs";
            return RTPN_ENOMEM;
        }
        cudaMemcpyAsync(snap, ctx->u, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        const int otx = ctx->tx, oty = ctx->ty, otz = ctx->tz, oc = ctx->depth;
        int rc = sweep(
            ctx->stream, reps, cands,
            [&](Tile t) { return rtpn_set_kernel_ex(ctx, kernel, t.x, t.y, t.z, t.c); },
            [&](cudaStream_t) {
                int r = rtpn_substep(ctx, 0, 0);
                return r ? r : rtpn_substep(ctx, 1, 0);
            },
            &best, &best_ms);
        cudaMemcpyAsync(ctx->u, snap, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        cudaFree(snap);
        if (rc) {
            rtpn_set_kernel_ex(ctx, kernel, otx, oty, otz, oc);
            return rc;
        }
        std::lock_guard<std::mutex> lock(g_mu);
        g_cache[key] = {best, best_ms};
        store_file(key, best, best_ms);
    }
    int rc = rtpn_set_kernel_ex(ctx, kernel, best.x, best.y, best.z, best.c);
    if (rc) return rc;
    if (tile) {
        tile[0] = best.x;
        tile[1] = best.y;
        tile[2] = best.z;
    }
    if (ms_per_step) *ms_per_step = best_ms;
    return RTPN_OK;
}

int rtpn_batch_autotune(rtpn_batch* b, int reps, int tile[3], double* ms_per_step) {
    if (!b || reps < 1) return RTPN_EINVAL;
    const int n = rtpn_batch_count(b);
    std::ostringstream k;
    k << "batch";
    std::vector<rtpn_ctx*> ctxs;
    for (int i = 0; i < n; ++i) {
        rtpn_ctx* c = rtpn_batch_instance(b, i);
        if (!c->media_set) return RTPN_ESTATE;
        ctxs.push_back(c);
        k << " " << c->N << ":" << c->g.nx << "x" << c->g.ny << "x" << c->g.nz << ":" << c->g.bc;
    }
    k << " prec=" << ctxs[0]->prec << " dev=" << device_key();
    const std::string key = k.str();
    Tile best{};
    rtpn_batch_get_tile(b, &best.x, &best.y, &best.z);
    double best_ms = -1.0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        load_file();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            best = it->second.first;
            best_ms = it->second.second;
        }
    }
    if (best_ms < 0) {
        size_t bytes = 0;
        for (auto* c : ctxs) bytes += (size_t)c->md.nc * c->g.V * c->elem;
        char* snap = nullptr;
        if (cudaMalloc(&snap, bytes) != cudaSuccess) {
            cudaGetLastError();
            return RTPN_ENOMEM;
        }
        cudaStream_t st = ctxs[0]->stream;
        std::vector<long long> done;
        for (auto* c : ctxs) done.push_back(c->steps_done);
        size_t off = 0;
        for (auto* c : ctxs) {
            const size_t nb = (size_t)c->md.nc * c->g.V * c->elem;
            cudaMemcpyAsync(snap + off, c->u, nb, cudaMemcpyDeviceToDevice, st);
            off += nb;
        }
        Tile old = best;
        const std::vector<Tile> cands(std::begin(kCandidates), std::end(kCandidates));
        int rc = sweep(
            st, reps, cands, [&](Tile t) { return rtpn_batch_set_tile(b, t.x, t.y, t.z); },
            [&](cudaStream_t) { return rtpn_batch_step(b, 1); }, &best, &best_ms);
        off = 0;
        for (size_t i = 0; i < ctxs.size(); ++i) {
            rtpn_ctx* c = ctxs[i];
            const size_t nb = (size_t)c->md.nc * c->g.V * c->elem;
            cudaMemcpyAsync(c->u, snap + off, nb, cudaMemcpyDeviceToDevice, st);
            c->steps_done = done[i];
            off += nb;
        }
        cudaStreamSynchronize(st);
        cudaFree(snap);
        if (rc) {
            rtpn_batch_set_tile(b, old.x, old.y, old.z);
            return rc;
        }
        std::lock_guard<std::mutex> lock(g_mu);
        g_cache[key] = {best, best_ms};
        store_file(key, best, best_ms);
    }
    int rc = rtpn_batch_set_tile(b, best.x, best.y, best.z);
    if (rc) return rc;
    if (tile) {
        tile[0] = best.x;
        tile[1] = best.y;
        tile[2] = best.z;
    }
    if (ms_per_step) *ms_per_step = best_ms;
    return RTPN_OK;
}

}  // extern "C"
