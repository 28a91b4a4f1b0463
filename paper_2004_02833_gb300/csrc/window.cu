// One compiled variant of the register-window substep kernel: order RTPN_WN, target class
// RTPN_WCLS.  The build compiles this file once per variant (each gets its own __constant__ table,
// at most 64 KB); kernels_window.cu dispatches to them.
#include "window_impl.cuh"

#if !defined(RTPN_WN) || !defined(RTPN_WCLS)
#error "compile with -DRTPN_WN=<order> -DRTPN_WCLS=<0|1>"
#endif

#define RTPN_CAT2(a, b, c, d) a##_##b##_##c##_##d
#define RTPN_CAT(a, b, c, d) RTPN_CAT2(a, b, c, d)
#define RTPN_VARIANT(name) RTPN_CAT(name, N, RTPN_WN, RTPN_WCLS)

namespace rtpn {
namespace win {

// Internal linkage for everything but the uniquely named entry points: every variant of this file
// defines a kernel of the same name, and the linker must not merge them.
namespace {

constexpr int kN = RTPN_WN;
constexpr int kA = RTPN_WCLS;
constexpr int kSources = class_size(kN, 1 - kA);
static_assert(kSources * 10 * 4 <= 64 * 1024 - 1024, "coefficient table exceeds constant memory");

// coefficient of source j (class 1 - kA, local index) for relation k: M_d[a][b] * dir
__constant__ float c_coef[kSources * 10];

template <typename S, bool SCALED, bool ANISO>
__global__ void __launch_bounds__(256) k_window(Args a) {
    int x, y, z;
    if (!cell_of(a, blockIdx.x, threadIdx.x, &x, &y, &z)) return;
    substep_cell<kN, kA, S, SCALED, ANISO>(a, c_coef, x, y, z);
}

template <bool SCALED, bool ANISO>
int launch_form(int precision, const Args& a, cudaStream_t st) {
    const int threads = a.tx * a.ty * a.tz;
    const unsigned blocks = (unsigned)a.ntx * a.nty * a.ntz;
    if (precision == RTPN_BF16)
        k_window<__nv_bfloat16, SCALED, ANISO><<<blocks, threads, 0, st>>>(a);
    else
        k_window<float, SCALED, ANISO><<<blocks, threads, 0, st>>>(a);
    return (int)cudaGetLastError();
}

// the form a launch needs; the non-cubic and anisotropic forms exist up to kExtendedMaxN (a
// template, so that the discarded branch is not instantiated for larger orders)
template <int NN>
int launch_any(int precision, const Args& a, cudaStream_t st) {
    const bool scaled = a.sy != 1.f || a.sz != 1.f;
    if (scaled || a.aniso) {
        if constexpr (NN <= kExtendedMaxN) {
            if (scaled && a.aniso) return launch_form<true, true>(precision, a, st);
            if (scaled) return launch_form<true, false>(precision, a, st);
            return launch_form<false, true>(precision, a, st);
        } else {
            return (int)cudaErrorNotSupported;
        }
    }
    return launch_form<false, false>(precision, a, st);
}

}  // namespace

int RTPN_VARIANT(window_upload)(const float* host, int count) {
    if (count != kSources * 10) return (int)cudaErrorInvalidValue;
    return (int)cudaMemcpyToSymbol(c_coef, host, sizeof(float) * count);
}

int RTPN_VARIANT(window_launch)(int precision, const Args& a, cudaStream_t st) {
    return launch_any<kN>(precision, a, st);
}

}  // namespace win
}  // namespace rtpn
