// One compiled variant of the fused step kernel: order RTPN_FN.  The build compiles this file once
// per order listed in fused_variants.h (each with its own __constant__ tables); kernels_fused.cu
// dispatches to them.
#include "fused_impl.cuh"

#if !defined(RTPN_FN)
#error "compile with -DRTPN_FN=<order>"
#endif

#define RTPN_FCAT2(a, b, c) a##_##b##_##c
#define RTPN_FCAT(a, b, c) RTPN_FCAT2(a, b, c)
#define RTPN_FVARIANT(name) RTPN_FCAT(name, N, RTPN_FN)

namespace rtpn {
namespace fus {

// Internal linkage for everything but the uniquely named entry points (every variant defines a
// kernel of the same name).
namespace {

constexpr int kN = RTPN_FN;
constexpr int kNE = class_size(kN, 0);
constexpr int kNO = class_size(kN, 1);
constexpr int kRing = ring_bytes(kN);
static_assert((kNE + kNO) * 10 * 4 <= 64 * 1024 - 1024, "coefficient tables exceed constant memory");
static_assert(kRing <= 227 * 1024, "the ring of new even planes exceeds shared memory");

// coefficients M_d[a][b] * dir: even targets by odd source (c_coef_e), odd targets by even source
__constant__ float c_coef_e[kNO * 10];
__constant__ float c_coef_o[kNE * 10];

// two CTAs per SM where two rings fit the SM's shared memory (N <= 7)
constexpr int kMinBlocks = 2 * (kRing + 1024) <= 228 * 1024 ? 2 : 1;

template <typename S>
__global__ void __launch_bounds__(THREADS, kMinBlocks) k_fused(Args a) {
    extern __shared__ __align__(16) float ring[];
    const Tile t = tile_of(a, blockIdx.x);
    const int tid = threadIdx.x;
    even_phase<kN, S>(a, c_coef_e, ring, t, tid, t.z0 - 1);
    even_phase<kN, S>(a, c_coef_e, ring, t, tid, t.z0);
    for (int p = t.z0; p < t.z1; ++p) {
        even_phase<kN, S>(a, c_coef_e, ring, t, tid, p + 1);
        __syncthreads();
        odd_phase<kN, S>(a, c_coef_o, ring, t, tid, p);
        __syncthreads();
    }
}

template <typename S>
int launch_typed(Args a, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_fused<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRing);
    if (e != cudaSuccess) return (int)e;
    if (a.zc <= 0) {
        // at most one wave of resident CTAs: every chunk recomputes two planes of new even values
        // beyond its own, so fewer, longer chunks win as long as the wave is nearly full (P7 128^3
        // on a GB300: 0.87 ms per step with 32-plane chunks, 0.90 with 16, 0.93 with 8)
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<S>, THREADS, kRing);
        if (e != cudaSuccess) return (int)e;
        const long long xy = (long long)a.ntx * a.nty;
        long long chunks = (long long)sms * (per_sm > 0 ? per_sm : 1) / xy;
        const long long most = (a.nz + 3) / 4;
        if (chunks > most) chunks = most;
        if (chunks < 1) chunks = 1;
        a.zc = (int)((a.nz + chunks - 1) / chunks);
    }
    a.nzc = (a.nz + a.zc - 1) / a.zc;
    const long long blocks = (long long)a.ntx * a.nty * a.nzc;
    if (blocks > 0x7fffffffll) return (int)cudaErrorInvalidConfiguration;
    k_fused<S><<<(unsigned)blocks, THREADS, kRing, st>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace

int RTPN_FVARIANT(fused_upload)(const float* even_targets, int ne, const float* odd_targets, int no) {
    if (ne != kNO * 10 || no != kNE * 10) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbol(c_coef_e, even_targets, sizeof(float) * ne);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_coef_o, odd_targets, sizeof(float) * no);
    return (int)e;
}

int RTPN_FVARIANT(fused_launch)(int precision, const Args& a, cudaStream_t st) {
    return precision == RTPN_BF16 ? launch_typed<__nv_bfloat16>(a, st) : launch_typed<float>(a, st);
}

}  // namespace fus
}  // namespace rtpn
