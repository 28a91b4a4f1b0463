// Internal declarations shared by the C-ABI layer and the kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "model.h"
#include "rtpn.h"

namespace rtpn {

// ---- factor planes: per-cell FP64-computed substep factors, stored in the math precision ----
// Eq. (5) rearranged: u' = alpha u + beta r with alpha = exp(-c tau), beta = tau E(-c tau).
// Planes are [plane][cell]; slot code g = (gx-1) + 2(gy-1) + 4(gz-1).
constexpr int FAC_FULL = 0;    // tau = dt:   alpha at 2g, beta at 2g+1          (planes 0..15)
constexpr int FAC_HALF = 16;   // tau = dt/2: alpha at 16+2g, beta at 17+2g      (planes 16..31)
constexpr int FAC_U0 = 32;     // u_0 (c = sigma_a), tau = dt: alpha, beta, beta*q (planes 32..34)
constexpr int FAC_PLANES = 35;
// Anisotropic scattering (generic kernel only): after the 35 planes above, alpha and beta of every
// (slot code g, order l) at tau = dt, then the same at tau = dt/2 (offset aniso_half_ofs(N)).
__host__ __device__ constexpr int aniso_plane(int N, int g, int l) { return FAC_PLANES + 2 * (g * (N + 1) + l); }
__host__ __device__ constexpr int aniso_half_ofs(int N) { return 16 * (N + 1); }
__host__ __device__ inline int aniso_planes(int N) { return FAC_PLANES + 32 * (N + 1); }

struct Geom {
    int nx, ny, nz;
    long long V;   // cells
    int bc;        // RTPN_BC_*
    double h;      // cell size along x (the kernels' 1/h)
    double hy = 0, hz = 0;  // cell sizes along y and z (equal to h for cubic cells)
};

// cell size along axis 0 (x), 1 (y) or 2 (z)
inline double axis_h(const Geom& g, int axis) { return axis == 0 ? g.h : axis == 1 ? g.hy : g.hz; }
inline bool cubic_cells(const Geom& g) { return g.hy == g.h && g.hz == g.h; }

template <typename F>
struct PartnerTable {
    const int* row;     // [na + 1] offsets into the entries
    const int* src;     // internal source index
    const F* coef;      // M_d[a][b] / h, negated when the target reads its lower neighbour
    const int* code;    // axis * 2 + (1 if the neighbour is i + 1 else 0)
    const int* fplane;  // per target: plane of alpha (beta = next plane), FAC_U0 for u_0
    int a0, na;         // first internal target, count
};

// host copies of the partner table of one class (built from the Model)
struct HostTable {
    std::vector<int> row, src, code, fplane;
    std::vector<double> coef;
    int a0 = 0, na = 0;
};

// message for rtpn_last_error(NULL) (entry points without a context)
void note_error(const std::string& msg);

// ---- generic kernels (kernels_generic.cu) ----
template <typename S, typename F>
void launch_substep_generic(S* u, const F* fac, const PartnerTable<F>& tab, const Geom& g,
                            int fac_ofs, cudaStream_t st);
// scat: f_l (l = 0..N, device) of anisotropic scattering, or nullptr (isotropic: 35 planes only)
template <typename F>
void launch_media_factors(const double* sa, const double* ss, const double* q, F* fac,
                          const Geom& g, double dt, const double* scat, int N, cudaStream_t st);
template <typename Sin, typename Sout>
void launch_convert(const Sin* in, Sout* out, long long n, cudaStream_t st);
template <typename S>
void launch_sum(const S* x, long long n, double* partial, int nblocks, double* out, cudaStream_t st);
template <typename S>
void launch_count_nonfinite(const S* x, long long n, unsigned long long* out, cudaStream_t st);
constexpr int SUM_BLOCKS = 1024;

// ---- register-window kernels (kernels_window*.cu) ----
struct WindowLaunch {
    void* u;                // state (float or bf16), internal order
    const float* fac;       // factor planes
    Geom g;
    int cls;                // target class
    int fac_ofs;            // FAC_FULL or FAC_HALF (anisotropic: 0 or aniso_half_ofs(N))
    int tx, ty, tz;         // CTA tile
    bool aniso = false;     // per-order factor planes (anisotropic scattering)
};
// returns false if (N, precision) is not compiled in
bool window_supported(int N, int precision);
bool window_extended(int N);  // the window kernel's non-cubic and anisotropic forms are compiled for N
// uploads the coefficient constants of order N (idempotent); returns cudaError_t
int window_prepare(const Model& md, double h, int precision);
int launch_window(int N, int precision, const WindowLaunch& w, cudaStream_t st);

// ---- fused step kernels (kernels_fused.cu, fused.cu) ----
// One pass of the even full step and the odd step after it, from state x into state y (another
// buffer of the same layout).
struct FusedLaunch {
    const void* x;          // state before the pass
    void* y;                // state after the pass
    const float* fac;       // factor planes
    Geom g;
    int fac_odd;            // FAC_FULL or FAC_HALF for the odd step
    int zc;                 // planes per z chunk (0 = automatic)
};
bool fused_supported(int N, int precision);
// uploads the coefficient constants of order N (idempotent); returns cudaError_t
int fused_prepare(const Model& md, int precision);
int launch_fused(int N, int precision, const FusedLaunch& f, cudaStream_t st);

// transposed partner table (adjoint.cu): targets of class clsB, sources of the other class
HostTable transposed_table(const Model& md, int clsB, const Geom& g);

// ---- TMA-staged kernels (kernels_stage.cu, stage.cu) ----
// nx must give 16-byte rows for the tensor maps
bool stage_supported(int N, int precision, int nx);
bool stage_has_tile(int N, int tx, int ty, int tz, int depth, int precision);
// builds the tensor maps (tile 0,0,0 = default; depth 0 = any) and the coupling tables;
// returns cudaError_t
int stage_prepare(rtpn_ctx* ctx, int tx, int ty, int tz, int depth);
// compiled (tx, ty, tz, depth) of order N that fit for this precision into tiles[4*i..];
// returns the count
int stage_variants_of(int N, int precision, int* tiles, int max);
int launch_stage(rtpn_ctx* ctx, int cls, int fac_ofs, cudaStream_t st, long long skip_stage,
                 long long wait_limit);
// The transposed coupling of a substep for the adjoint's multipliers on the staged kernel:
// lam_B <- alpha_B lam_B + (1/h) K w_A (class B = tgt_cls; w: the w_planes planes of the other class,
// local order; alpha_B the factors at offset fac_ofs (FAC_FULL / FAC_HALF; u_0: its own), or 1 for
// fac_ofs < 0).  FP32 contexts with the staged kernel prepared; returns cudaError_t.
int launch_stage_adjoint_sources(rtpn_ctx* ctx, int tgt_cls, float* lam, const float* w, int w_planes,
                                 int fac_ofs, cudaStream_t st);
// The tensor maps of the staged kernel over another FP32 state (an adjoint segment's state) into
// maps_dev (device, stage_maps_bytes(ctx) bytes, 128-byte aligned); returns cudaError_t.
size_t stage_maps_bytes(const rtpn_ctx* ctx);
int stage_maps_for(rtpn_ctx* ctx, const void* state, void* maps_dev);
// A forward pass on class cls between FP32 states: sources through src_maps, the old targets
// through the plane maps that start tgt_maps (both from stage_maps_for), the new targets into out
// (full state layout; only class cls is written).  Returns cudaError_t.
int launch_stage_between(rtpn_ctx* ctx, int cls, int fac_ofs, const void* src_maps, const void* tgt_maps,
                         void* out, cudaStream_t st);
constexpr long long STAGE_WAIT_LIMIT = 1ll << 20;  // mbarrier polls (each <= 2 us) before a wait gives up

}  // namespace rtpn

struct rtpn_ctx {
    rtpn::Model md;
    rtpn::Geom g{};
    int N = 0, prec = RTPN_FP32, kernel = RTPN_KERNEL_AUTO, active_kernel = RTPN_KERNEL_GENERIC;
    int tx = 0, ty = 0, tz = 0;
    int depth = 0;                   // stage buffers of the staged kernel, 0 = any
    double dt = 0;
    size_t elem = 4;                 // bytes per stored moment
    void* u = nullptr;               // state [internal c][z][y][x]
    void* u_alt = nullptr;           // the fused kernel's second state buffer (swaps with u per pass)
    void* u_home = nullptr;          // the state buffer allocated at creation (fixed)
    void* fac = nullptr;             // factor planes (double for FP64, float otherwise)
    void* table_mem = nullptr;       // device partner tables (both classes)
    rtpn::PartnerTable<double> tab64[2]{};
    rtpn::PartnerTable<float> tab32[2]{};
    double* partial = nullptr;       // reduction partials [SUM_BLOCKS] + result
    unsigned long long* counter = nullptr;
    void* staging = nullptr;         // one plane of FP64 (conversions, media upload)
    double* media = nullptr;         // FP64 sigma_a, sigma_s, q as last set (3 planes)
    cudaStream_t stream = nullptr;   // work stream (user's or own)
    cudaStream_t own = nullptr;      // private stream (capture, default work stream)
    bool media_set = false;
    bool batch_member = false;       // created by rtpn_batch_create (its kernels take cubic cells)
    double* scat = nullptr;          // f_l (l = 0..N) of anisotropic scattering on the device, or null
    int fac_planes = rtpn::FAC_PLANES;  // factor planes allocated
    long long steps_done = 0;
    std::map<int, cudaGraphExec_t> graphs;  // pair-sequence graphs keyed by pair count
    std::string err;
    unsigned* status = nullptr;      // device status words: [0] bounded-wait / check bits, [1..7] record
    void* stage_mem = nullptr;       // staged kernels: coupling tables of both classes + column starts
    size_t stage_tab_bytes[2] = {0, 0};
    int stage_variant = -1, sms = 0;
    bool tile_from_stage = false;    // tx, ty, tz, depth describe the staged variant in use (not a request)
    void* stage_maps_dev = nullptr;  // CUtensorMap of the staged kernel (device global memory): those over
                                     // u, then the adjoint's (over its w, then over its lam)
    const void* stage_adj_lam = nullptr;  // arrays the adjoint maps were built for
    const void* stage_adj_w = nullptr;
    // the staged FP32 adjoint's work buffers (checkpoints, segment states, multipliers, tensor maps
    // over them), kept between calls; rtpn_adjoint_release frees them
    void* adj_ws = nullptr;
    size_t adj_ws_bytes = 0;
    long long adj_maps_key[4] = {-1, -1, -1, -1};  // (segments, ring states, variant, workspace) of the maps
};
