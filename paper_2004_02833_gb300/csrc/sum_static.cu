// FP64 sum of a device array with scratch in a file-scope device array: this entry point allocates
// nothing.  The library has no counterpart of it in the paper; it exists for callers that cannot
// call cudaMalloc at the point where they need the sum.
#include <mutex>
#include <string>

#include "rtpn_internal.h"

namespace rtpn {
namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = (long long)kThreads * 64;        // elements summed per partial
constexpr int kMaxPartials = 1 << 16;                          // 512 KB of FP64 partials
constexpr long long kMaxElems = kChunk * (long long)kMaxPartials;  // 2^30 elements

// Shared by every call on a device and kept until the process exits.  Each call overwrites the
// partials it uses before reading them, so nothing has to start at zero.
static __device__ __align__(256) double g_sum_scratch[kMaxPartials];

template <typename T>
__device__ __forceinline__ double as_f64(T v) { return (double)v; }

// partial[b] = sum of x[b*kChunk .. min(n, (b+1)*kChunk)) in a fixed order
template <typename T>
__global__ void k_chunk_sums(const T* __restrict__ x, long long n, double* __restrict__ partial) {
    const long long begin = (long long)blockIdx.x * kChunk;
    const long long end = begin + kChunk < n ? begin + kChunk : n;
    double acc = 0.0;
    for (long long i = begin + threadIdx.x; i < end; i += kThreads) acc += as_f64(x[i]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double ws[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += ws[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void k_chunks_total(const double* __restrict__ partial, int count, double* __restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
        *out = s;
    }
}

// The driver's current context, through the runtime's entry-point query (no link to libcuda).
typedef int (*CtxGetCurrentFn)(void** ctx);
CtxGetCurrentFn ctx_get_current() {
    static std::once_flag once;
    static CtxGetCurrentFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    });
    return fn;
}

// Device address of g_sum_scratch on the current device, looked up once per device and context
// (the set-up): a device reset or a new primary context gets a fresh lookup, never a stale address.
int scratch_address(double** out) {
    static std::mutex mu;
    static double* addr[256] = {};
    static void* owner[256] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= 256) return (int)cudaErrorInvalidDevice;
    CtxGetCurrentFn get = ctx_get_current();
    if (!get) return (int)cudaErrorDeviceUninitialized;
    void* cur = nullptr;
    if (get(&cur) != 0) return (int)cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lock(mu);
    if (!cur || !addr[dev] || owner[dev] != cur) {
        // the lookup also makes the device's primary context current on this thread
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sum_scratch);
        if (e != cudaSuccess) return (int)e;
        if (get(&cur) != 0 || !cur) return (int)cudaErrorDeviceUninitialized;
        addr[dev] = (double*)p;
        owner[dev] = cur;
    }
    *out = addr[dev];
    return 0;
}

}  // namespace
}  // namespace rtpn

extern "C" int rtpn_sum_static(const void* x, int dtype, long long n, double* out, void* stream) {
    using namespace rtpn;
    if (!out || n < 0 || (n > 0 && !x) || (dtype != RTPN_DTYPE_F64 && dtype != RTPN_DTYPE_F32)) {
        note_error("rtpn_sum_static: bad argument");
        return RTPN_EINVAL;
    }
    if (n > kMaxElems) {
        note_error("rtpn_sum_static: n exceeds 2^30 elements, the capacity of its static scratch");
        return RTPN_EINVAL;
    }
    double* partial = nullptr;
    int rc = scratch_address(&partial);
    if (rc) {
        note_error(std::string("rtpn_sum_static: scratch address: ") +
                   cudaGetErrorString((cudaError_t)rc));
        return RTPN_ECUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int count = (int)((n + kChunk - 1) / kChunk);
    if (count > 0) {
        if (dtype == RTPN_DTYPE_F64)
            k_chunk_sums<double><<<count, kThreads, 0, st>>>((const double*)x, n, partial);
        else
            k_chunk_sums<float><<<count, kThreads, 0, st>>>((const float*)x, n, partial);
    }
    k_chunks_total<<<1, 1024, 0, st>>>(partial, count, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_error(std::string("rtpn_sum_static: launch: ") + cudaGetErrorString(e));
        return RTPN_ECUDA;
    }
    return RTPN_OK;
}
