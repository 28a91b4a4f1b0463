// One variant of the TMA-staged substep kernel: order RTPN_SN, CTA tile RTPN_STX x RTPN_STY x
// RTPN_STZ, RTPN_SNB stage buffers, TMA box lengths in multiples of RTPN_SEM components, both target
// classes, FP32 and BF16 storage.  kernels_stage.cu dispatches to it.
#include "stage_impl.cuh"

#if !defined(RTPN_SN) || !defined(RTPN_STX) || !defined(RTPN_STY) || !defined(RTPN_STZ) || !defined(RTPN_SNB) || \
    !defined(RTPN_SEM)
#error "compile with -DRTPN_SN=<order> -DRTPN_STX=.. -DRTPN_STY=.. -DRTPN_STZ=.. -DRTPN_SNB=.. -DRTPN_SEM=.."
#endif

#define RTPN_SCAT2(a, b, c, d, e, f, g) a##_##b##_##c##_##d##_##e##_##f##_##g
#define RTPN_SCAT(a, b, c, d, e, f, g) RTPN_SCAT2(a, b, c, d, e, f, g)
#define RTPN_SVARIANT(name) RTPN_SCAT(name, RTPN_SN, RTPN_STX, RTPN_STY, RTPN_STZ, RTPN_SNB, RTPN_SEM)

namespace rtpn {
namespace stg {

// Everything but the uniquely named entry points has internal linkage: every variant of this file
// defines a k_stage / launch_one of the same name, and the linker must not merge them.
namespace {

constexpr int kN = RTPN_SN, kTX = RTPN_STX, kTY = RTPN_STY, kTZ = RTPN_STZ, kNB = RTPN_SNB, kEM = RTPN_SEM;
constexpr int kThreads = Layout<kN, 0, float, kTX, kTY, kTZ, kNB, kEM>::THREADS;
// Two CTAs per SM where two rings fit shared memory and the order's window fits the registers
// that leaves (orders up to 15: about 110 registers a thread); one otherwise.
constexpr int kMinBlocks = (kN <= 15 && 2 * Layout<kN, 0, float, kTX, kTY, kTZ, kNB, kEM>::BYTES <= 232448) ? 2 : 1;

template <int A, typename S, int MODE>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_stage(Args a) {
    static_assert(Layout<kN, A, S, kTX, kTY, kTZ, kNB, kEM>::FITS, "stage ring exceeds shared memory");
    extern __shared__ __align__(128) unsigned char smem[];
    stage_kernel_body<kN, A, S, kTX, kTY, kTZ, kNB, kEM, MODE>(a, smem);
}

template <int A, typename S, int MODE>
int launch_one(const Args& a, int sms, cudaStream_t st) {
    using L = Layout<kN, A, S, kTX, kTY, kTZ, kNB, kEM>;
    if constexpr (!L::FITS) {
        return (int)cudaErrorNotSupported;  // this depth is compiled for the narrower storage only
    } else {
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_stage<A, S, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             L::BYTES);
        if (e != cudaSuccess) return (int)e;
        configured[dev] = true;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage<A, S, MODE>, kThreads, L::BYTES);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorLaunchOutOfResources;
    long long grid = (long long)per_sm * sms;
    if (grid > a.tiles) grid = a.tiles;
    if (grid < 1) return 0;
    k_stage<A, S, MODE><<<(unsigned)grid, kThreads, L::BYTES, st>>>(a);
    return (int)cudaGetLastError();
    }
}

// dynamic shared memory of the variant, or 0 if it does not fit a CTA
template <int A, typename S>
constexpr int smem_of() {
    using L = Layout<kN, A, S, kTX, kTY, kTZ, kNB, kEM>;
    return L::FITS ? L::BYTES : 0;
}
// box geometry of the variant for a storage precision (the host builds its tensor maps with it):
// out = {maps per kind, box length step, x halo group width, x halo group rows}
template <typename S>
void geom_of(int* out) {
    using L = Layout<kN, 0, S, kTX, kTY, kTZ, kNB, kEM>;
    out[0] = L::NMAP;
    out[1] = kEM;
    out[2] = L::XW;
    out[3] = L::RY;
}

}  // namespace

// mode FORWARD: FP32 or BF16 storage; mode ADJ_SOURCES: FP32 (the adjoint)
int RTPN_SVARIANT(stage_launch)(int cls, int precision, int mode, const Args& a, int sms, cudaStream_t st) {
    if (mode == ADJ_SOURCES) {
        if (precision != RTPN_FP32) return (int)cudaErrorNotSupported;
        return cls == 0 ? launch_one<0, float, ADJ_SOURCES>(a, sms, st) : launch_one<1, float, ADJ_SOURCES>(a, sms, st);
    }
    if (precision == RTPN_BF16)
        return cls == 0 ? launch_one<0, __nv_bfloat16, FORWARD>(a, sms, st)
                        : launch_one<1, __nv_bfloat16, FORWARD>(a, sms, st);
    return cls == 0 ? launch_one<0, float, FORWARD>(a, sms, st) : launch_one<1, float, FORWARD>(a, sms, st);
}

void RTPN_SVARIANT(stage_geom)(int precision, int* out) {
    if (precision == RTPN_BF16)
        geom_of<__nv_bfloat16>(out);
    else
        geom_of<float>(out);
}

int RTPN_SVARIANT(stage_smem)(int cls, int precision) {
    if (precision == RTPN_BF16) return cls == 0 ? smem_of<0, __nv_bfloat16>() : smem_of<1, __nv_bfloat16>();
    return cls == 0 ? smem_of<0, float>() : smem_of<1, float>();
}

}  // namespace stg
}  // namespace rtpn
