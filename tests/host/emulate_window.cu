// Host run of the register-window substep kernel's per-cell body (test program): every cell of the
// grid in turn, over bounds-checked memory (the program aborts on an access outside the state and
// factor buffers).  The factor planes follow the rule of rtpn_set_media (mean of sigma over the
// cells adjacent to a sub-grid point; alpha = exp(-c tau), beta = tau E(-c tau)).
//
// usage: emulate_window N cls nx ny nz bc h dt half fp32|bf16 in.bin out.bin [hy hz [g]]
//   in.bin: float64 u [n_c][nz][ny][nx] (interface order), then sigma_a, sigma_s, q [nz][ny][nx]
//   out.bin: float64 u after the substep of class cls (tau = dt, or dt/2 with half = 1)
//   hy hz: cell sizes along y and z (non-cubic cells: the body's scaled form), default h
//   g: anisotropic scattering with f_l = g^l (the body's anisotropic form, per-order factor planes)
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>
#include <string>

static const char* g_lo[4];
static const char* g_hi[4];
static int g_nr = 0;
static void check_ptr(const void* p) {
    const char* c = (const char*)p;
    for (int i = 0; i < g_nr; ++i) if (c >= g_lo[i] && c < g_hi[i]) return;
    fprintf(stderr, "OUT OF BOUNDS access %p\n", p);
    std::abort();
}
#define RTPN_HOST_CHECK 1
#define RTPN_CHECK_PTR(p) check_ptr(p)
#include "window_impl.cuh"

using namespace rtpn;

template <int N, int A, typename S, bool SC, bool AN>
void run(const win::Args& a, const float* coef) {
    for (int z = 0; z < a.nz; ++z)
        for (int y = 0; y < a.ny; ++y)
            for (int x = 0; x < a.nx; ++x) win::substep_cell<N, A, S, SC, AN>(a, coef, x, y, z);
}

template <typename S, bool SC, bool AN>
void dispatch_form(int N, int A, const win::Args& a, const float* coef) {
#define CASE(n) if (N == n) { if (A == 0) run<n, 0, S, SC, AN>(a, coef); else run<n, 1, S, SC, AN>(a, coef); return; }
    CASE(1) CASE(3) CASE(7) CASE(15)
#undef CASE
    fprintf(stderr, "N not compiled\n"); std::abort();
}

template <typename S>
void dispatch(int N, int A, const win::Args& a, const float* coef) {
    const bool sc = a.sy != 1.f || a.sz != 1.f;
    if (sc && a.aniso)
        dispatch_form<S, true, true>(N, A, a, coef);
    else if (sc)
        dispatch_form<S, true, false>(N, A, a, coef);
    else if (a.aniso)
        dispatch_form<S, false, true>(N, A, a, coef);
    else
        dispatch_form<S, false, false>(N, A, a, coef);
}

int main(int argc, char** argv) {
    if (argc < 12) { fprintf(stderr, "usage\n"); return 2; }
    int N = atoi(argv[1]), A = atoi(argv[2]), nx = atoi(argv[3]), ny = atoi(argv[4]), nz = atoi(argv[5]);
    int bc = atoi(argv[6]); double h = atof(argv[7]), dt = atof(argv[8]); int half = atoi(argv[9]);
    std::string prec = argv[10];
    const char* inf = argv[11]; const char* outf = argv[12];
    const double hy = argc > 14 ? atof(argv[13]) : h, hz = argc > 14 ? atof(argv[14]) : h;
    const bool aniso = argc > 15;
    const double gscat = aniso ? atof(argv[15]) : 0.0;
    Model md = build_model(N);
    long long V = (long long)nx * ny * nz;
    std::vector<double> in((size_t)(md.nc + 3) * V);
    FILE* f = fopen(inf, "rb");
    if (!f || fread(in.data(), 8, in.size(), f) != in.size()) { fprintf(stderr, "bad input\n"); return 4; }
    fclose(f);
    const double* sa = in.data() + (size_t)md.nc * V; const double* ss = sa + V; const double* q = ss + V;
    // factors (same rule as the device precompute)
    std::vector<float> fac((size_t)(aniso ? aniso_planes(N) : FAC_PLANES) * V);
    auto idx = [&](int x, int y, int z) { return ((long long)z * ny + y) * nx + x; };
    for (int z = 0; z < nz; ++z) for (int y = 0; y < ny; ++y) for (int x = 0; x < nx; ++x) {
        long long cell = idx(x, y, z);
        for (int code = 0; code < 8; ++code) {
            int gx = code & 1, gy = (code >> 1) & 1, gz = (code >> 2) & 1;
            double sum = 0, sum_a = 0, sum_s = 0; int cnt = 0;
            for (int dz = 0; dz <= gz; ++dz) for (int dy = 0; dy <= gy; ++dy) for (int dx = 0; dx <= gx; ++dx) {
                int xx = x + dx, yy = y + dy, zz = z + dz;
                if (xx >= nx || yy >= ny || zz >= nz) { if (bc) continue; xx %= nx; yy %= ny; zz %= nz; }
                long long j = idx(xx, yy, zz); sum += sa[j] + ss[j]; sum_a += sa[j]; sum_s += ss[j]; ++cnt;
            }
            double c = sum / cnt;
            // per order l with anisotropic scattering: c_l = sigma_a + (1 - f_l) sigma_s (point means)
            for (int l = 0; aniso && l <= N; ++l) {
                const double cl = (sum_a + (1.0 - std::pow(gscat, l)) * sum_s) / cnt;
                for (int hh = 0; hh < 2; ++hh) {
                    const double tau = hh ? 0.5 * dt : dt;
                    const double al = exp(-cl * tau), be = cl != 0 ? -expm1(-cl * tau) / cl : tau;
                    const size_t pl = (size_t)(aniso_plane(N, code, l) + (hh ? aniso_half_ofs(N) : 0));
                    fac[pl * V + cell] = (float)al;
                    fac[(pl + 1) * V + cell] = (float)be;
                }
            }
            for (int hh = 0; hh < 2; ++hh) {
                double tau = hh ? 0.5 * dt : dt;
                double al = exp(-c * tau), be = c > 0 ? -expm1(-c * tau) / c : tau;
                fac[(size_t)((hh ? FAC_HALF : FAC_FULL) + 2 * code) * V + cell] = (float)al;
                fac[(size_t)((hh ? FAC_HALF : FAC_FULL) + 2 * code + 1) * V + cell] = (float)be;
            }
        }
        double c = sa[cell], al = exp(-c * dt), be = c > 0 ? -expm1(-c * dt) / c : dt;
        fac[(size_t)FAC_U0 * V + cell] = (float)al; fac[(size_t)(FAC_U0 + 1) * V + cell] = (float)be;
        fac[(size_t)(FAC_U0 + 2) * V + cell] = (float)(be * q[cell]);
    }
    std::vector<float> coef;
    if (!win::coef_table(md, A, &coef)) { fprintf(stderr, "coef table mismatch\n"); return 3; }
    win::Args a{};
    a.fac = fac.data(); a.V = V; a.nx = nx; a.ny = ny; a.nz = nz; a.bc = bc;
    a.fac_ofs = aniso ? (half ? aniso_half_ofs(N) : 0) : (half ? FAC_HALF : FAC_FULL); a.inv_h = (float)(1.0 / h);
    a.aniso = aniso ? 1 : 0;
    a.sy = (float)(h / hy); a.sz = (float)(h / hz);
    a.tx = a.ty = a.tz = 1; a.ntx = nx; a.nty = ny; a.ntz = nz;
    g_lo[0] = (const char*)fac.data(); g_hi[0] = (const char*)(fac.data() + fac.size());
    std::vector<double> out((size_t)md.nc * V);
    if (prec == "fp32") {
        std::vector<float> u((size_t)md.nc * V);
        for (int c = 0; c < md.nc; ++c) for (long long i = 0; i < V; ++i)
            u[(size_t)md.internal_of_abi[c] * V + i] = (float)in[(size_t)c * V + i];
        g_lo[1] = (const char*)u.data(); g_hi[1] = (const char*)(u.data() + u.size()); g_nr = 2;
        a.u = u.data();
        dispatch<float>(N, A, a, coef.data());
        for (int c = 0; c < md.nc; ++c) for (long long i = 0; i < V; ++i)
            out[(size_t)c * V + i] = u[(size_t)md.internal_of_abi[c] * V + i];
    } else {
        std::vector<__nv_bfloat16> u((size_t)md.nc * V);
        for (int c = 0; c < md.nc; ++c) for (long long i = 0; i < V; ++i)
            u[(size_t)md.internal_of_abi[c] * V + i] = __float2bfloat16_rn((float)in[(size_t)c * V + i]);
        g_lo[1] = (const char*)u.data(); g_hi[1] = (const char*)(u.data() + u.size()); g_nr = 2;
        a.u = u.data();
        dispatch<__nv_bfloat16>(N, A, a, coef.data());
        for (int c = 0; c < md.nc; ++c) for (long long i = 0; i < V; ++i)
            out[(size_t)c * V + i] = __bfloat162float(u[(size_t)md.internal_of_abi[c] * V + i]);
    }
    f = fopen(outf, "wb"); fwrite(out.data(), 8, out.size(), f); fclose(f);
    return 0;
}
