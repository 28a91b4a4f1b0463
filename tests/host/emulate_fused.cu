// Host run of the fused step kernel's phases (test program): the CTAs and their threads run one after
// another, with the kernel's barriers as phase boundaries, over bounds-checked memory (every global
// access must fall in the state, output or factor buffers, every ring access in the CTA's ring;
// the program aborts otherwise).  The factor planes follow the rule of rtpn_set_media (mean of
// sigma over the cells adjacent to a sub-grid point; alpha = exp(-c tau), beta = tau E(-c tau)).
//
// usage: emulate_fused N zc nx ny nz bc h dt half fp32|bf16 in.bin out.bin
//   in.bin: float64 u [n_c][nz][ny][nx] (interface order), then sigma_a, sigma_s, q [nz][ny][nx]
//   out.bin: float64 u after one fused pass (even full step, odd step with dt or dt/2)
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
static const float* g_rlo; static const float* g_rhi;
static void check_ring(const float* p) {
    if (p < g_rlo || p >= g_rhi) { fprintf(stderr, "RING OUT OF BOUNDS %ld\n", (long)(p - g_rlo)); std::abort(); }
}
#define RTPN_HOST_CHECK 1
#define RTPN_CHECK_PTR(p) check_ptr(p)
#define RTPN_CHECK_RING(p) check_ring(p)
#include "fused_impl.cuh"

using namespace rtpn;

template <int N, typename S>
void run(fus::Args a, const float* ce, const float* co) {
    std::vector<float> ring(fus::ring_bytes(N) / 4, NAN);
    g_rlo = ring.data(); g_rhi = ring.data() + ring.size();
    const int blocks = a.ntx * a.nty * a.nzc;
    for (int b = 0; b < blocks; ++b) {
        std::fill(ring.begin(), ring.end(), NAN);
        const fus::Tile t = fus::tile_of(a, b);
        for (int tid = 0; tid < fus::THREADS; ++tid) fus::even_phase<N, S>(a, ce, ring.data(), t, tid, t.z0 - 1);
        for (int tid = 0; tid < fus::THREADS; ++tid) fus::even_phase<N, S>(a, ce, ring.data(), t, tid, t.z0);
        for (int p = t.z0; p < t.z1; ++p) {
            for (int tid = 0; tid < fus::THREADS; ++tid) fus::even_phase<N, S>(a, ce, ring.data(), t, tid, p + 1);
            for (int tid = 0; tid < fus::THREADS; ++tid) fus::odd_phase<N, S>(a, co, ring.data(), t, tid, p);
        }
    }
}

template <typename S>
void dispatch(int N, const fus::Args& a, const float* ce, const float* co) {
#define CASE(n) if (N == n) { run<n, S>(a, ce, co); return; }
    CASE(1) CASE(3) CASE(5) CASE(7) CASE(9)
    fprintf(stderr, "N not compiled\n"); std::abort();
}

int main(int argc, char** argv) {
    if (argc < 12) { fprintf(stderr, "usage\n"); return 2; }
    int N = atoi(argv[1]), zc = atoi(argv[2]), nx = atoi(argv[3]), ny = atoi(argv[4]), nz = atoi(argv[5]);
    int bc = atoi(argv[6]); double h = atof(argv[7]), dt = atof(argv[8]); int half = atoi(argv[9]);
    std::string prec = argv[10];
    const char* inf = argv[11]; const char* outf = argv[12];
    Model md = build_model(N);
    long long V = (long long)nx * ny * nz;
    std::vector<double> in((size_t)(md.nc + 3) * V);
    FILE* f = fopen(inf, "rb"); if (fread(in.data(), 8, in.size(), f) != in.size()) return 4; fclose(f);
    const double* sa = in.data() + (size_t)md.nc * V; const double* ss = sa + V; const double* q = ss + V;
    std::vector<float> fac((size_t)FAC_PLANES * V);
    auto idx = [&](int x, int y, int z) { return ((long long)z * ny + y) * nx + x; };
    for (int z = 0; z < nz; ++z) for (int y = 0; y < ny; ++y) for (int x = 0; x < nx; ++x) {
        long long cell = idx(x, y, z);
        for (int code = 0; code < 8; ++code) {
            int gx = code & 1, gy = (code >> 1) & 1, gz = (code >> 2) & 1;
            double sum = 0; int cnt = 0;
            for (int dz = 0; dz <= gz; ++dz) for (int dy = 0; dy <= gy; ++dy) for (int dx = 0; dx <= gx; ++dx) {
                int xx = x + dx, yy = y + dy, zz = z + dz;
                if (xx >= nx || yy >= ny || zz >= nz) { if (bc) continue; xx %= nx; yy %= ny; zz %= nz; }
                long long j = idx(xx, yy, zz); sum += sa[j] + ss[j]; ++cnt;
            }
            double c = sum / cnt;
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
    std::vector<float> ce, co;
    if (!win::coef_table(md, 0, &ce) || !win::coef_table(md, 1, &co)) { fprintf(stderr, "coef table mismatch\n"); return 3; }
    fus::Args a{};
    a.fac = fac.data(); a.V = V; a.nx = nx; a.ny = ny; a.nz = nz; a.bc = bc;
    a.fac_even = FAC_FULL; a.fac_odd = half ? FAC_HALF : FAC_FULL; a.inv_h = (float)(1.0 / h);
    a.zc = zc; a.ntx = (nx + fus::TX - 1) / fus::TX; a.nty = (ny + fus::TY - 1) / fus::TY; a.nzc = (nz + zc - 1) / zc;
    g_lo[0] = (const char*)fac.data(); g_hi[0] = (const char*)(fac.data() + fac.size());
    std::vector<double> out((size_t)md.nc * V);
    auto go = [&](auto tag) {
        using S = decltype(tag);
        std::vector<S> u((size_t)md.nc * V), y((size_t)md.nc * V);
        for (auto& v : y) v = S(NAN);
        for (int c = 0; c < md.nc; ++c) for (long long i = 0; i < V; ++i)
            u[(size_t)md.internal_of_abi[c] * V + i] = S((float)in[(size_t)c * V + i]);
        g_lo[1] = (const char*)u.data(); g_hi[1] = (const char*)(u.data() + u.size());
        g_lo[2] = (const char*)y.data(); g_hi[2] = (const char*)(y.data() + y.size()); g_nr = 3;
        a.x = u.data(); a.y = y.data();
        dispatch<S>(N, a, ce.data(), co.data());
        for (int c = 0; c < md.nc; ++c) for (long long i = 0; i < V; ++i)
            out[(size_t)c * V + i] = (double)(float)y[(size_t)md.internal_of_abi[c] * V + i];
    };
    if (prec == "fp32") go(float{}); else go(__nv_bfloat16{});
    f = fopen(outf, "wb"); fwrite(out.data(), 8, out.size(), f); fclose(f);
    return 0;
}
