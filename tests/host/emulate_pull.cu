// Host run of the staged adjoint's per-cell arithmetic (test program): the factor derivatives
// (adj::factor_derivatives) and the pull-back through one pass from its stored pre- and post-pass
// states (adj::pull_cells, grouped by adj::pull_table), over every cell in groups of four, on
// bounds-checked memory (the program aborts on an access outside the arrays it was given).  The
// factor planes follow the rule of rtpn_set_media (mean of sigma over the cells adjacent to a
// sub-grid point; alpha = exp(-c tau), beta = tau E(-c tau)), FP32.
//
// usage: emulate_pull N cls nx ny nz bc h dt half pre in.bin out.bin
//   cls: the class of the pass; half: tau = dt/2; pre: -1, or a pending factor of the class at
//   dt (0) or dt/2 (1) applied first
//   in.bin: float64 upre [n_c], upost [n_c], lam [n_c] (interface order), sigma_a, sigma_s, q
//   out.bin: float64 w [n_c] (the class's components at their interface positions, 0 elsewhere),
//   lam [n_c] after, gacc [9][V], gq [V]
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

static const char* g_lo[16];
static const char* g_hi[16];
static int g_nr = 0;
static void check_ptr(const void* p) {
    const char* c = (const char*)p;
    for (int i = 0; i < g_nr; ++i)
        if (c >= g_lo[i] && c < g_hi[i]) return;
    fprintf(stderr, "OUT OF BOUNDS access %p\n", p);
    std::abort();
}
#define RTPN_HOST_CHECK 1
#define RTPN_CHECK_PTR(p) check_ptr(p)
#include "pull_impl.cuh"

using namespace rtpn;

template <typename T>
static void region(const std::vector<T>& v) {
    g_lo[g_nr] = (const char*)v.data();
    g_hi[g_nr] = (const char*)(v.data() + v.size());
    ++g_nr;
}

int main(int argc, char** argv) {
    if (argc < 13) {
        fprintf(stderr, "usage\n");
        return 2;
    }
    const int N = atoi(argv[1]), A = atoi(argv[2]), nx = atoi(argv[3]), ny = atoi(argv[4]), nz = atoi(argv[5]);
    const int bc = atoi(argv[6]);
    const double h = atof(argv[7]), dt = atof(argv[8]);
    const int half = atoi(argv[9]), pre = atoi(argv[10]);
    Model md = build_model(N);
    const long long V = (long long)nx * ny * nz;
    if (V % 4 != 0) {
        fprintf(stderr, "V must be a multiple of 4\n");
        return 2;
    }
    std::vector<double> in((size_t)(3 * md.nc + 3) * V);
    FILE* f = fopen(argv[11], "rb");
    if (!f || fread(in.data(), 8, in.size(), f) != in.size()) {
        fprintf(stderr, "bad input\n");
        return 4;
    }
    fclose(f);
    std::vector<double> sa(in.begin() + (size_t)3 * md.nc * V, in.begin() + (size_t)(3 * md.nc + 1) * V);
    std::vector<double> ss(in.begin() + (size_t)(3 * md.nc + 1) * V, in.begin() + (size_t)(3 * md.nc + 2) * V);
    const double* q = in.data() + (size_t)(3 * md.nc + 2) * V;
    Geom g{};
    g.nx = nx, g.ny = ny, g.nz = nz, g.V = V, g.bc = bc, g.h = h, g.hy = h, g.hz = h;
    // factor planes (alpha, beta per slot code at dt and dt/2; u_0's alpha, beta, beta q)
    std::vector<float> fac((size_t)FAC_PLANES * V);
    auto idx = [&](int x, int y, int z) { return ((long long)z * ny + y) * nx + x; };
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long long cell = idx(x, y, z);
                for (int code = 0; code < 8; ++code) {
                    const int gx = code & 1, gy = (code >> 1) & 1, gz = (code >> 2) & 1;
                    double sum = 0;
                    int cnt = 0;
                    for (int dz = 0; dz <= gz; ++dz)
                        for (int dy = 0; dy <= gy; ++dy)
                            for (int dx = 0; dx <= gx; ++dx) {
                                int xx = x + dx, yy = y + dy, zz = z + dz;
                                if (xx >= nx || yy >= ny || zz >= nz) {
                                    if (bc) continue;
                                    xx %= nx;
                                    yy %= ny;
                                    zz %= nz;
                                }
                                const long long j = idx(xx, yy, zz);
                                sum += sa[j] + ss[j];
                                ++cnt;
                            }
                    const double c = sum / cnt;
                    for (int hh = 0; hh < 2; ++hh) {
                        const double tau = hh ? 0.5 * dt : dt;
                        const double al = exp(-c * tau), be = c != 0 ? -expm1(-c * tau) / c : tau;
                        fac[(size_t)((hh ? FAC_HALF : FAC_FULL) + 2 * code) * V + cell] = (float)al;
                        fac[(size_t)((hh ? FAC_HALF : FAC_FULL) + 2 * code + 1) * V + cell] = (float)be;
                    }
                }
                const double c = sa[cell], al = exp(-c * dt), be = c != 0 ? -expm1(-c * dt) / c : dt;
                fac[(size_t)FAC_U0 * V + cell] = (float)al;
                fac[(size_t)(FAC_U0 + 1) * V + cell] = (float)be;
                fac[(size_t)(FAC_U0 + 2) * V + cell] = (float)(be * q[cell]);
            }
    std::vector<float> dfac((size_t)adj::DFAC_PLANES * V);
    region(sa);
    region(ss);
    region(dfac);
    for (long long cell = 0; cell < V; ++cell) adj::factor_derivatives<float>(sa.data(), ss.data(), dfac.data(), g, dt, cell);
    // the class's arrays: pre- and post-pass values and multipliers in internal order
    const int a0 = A == 0 ? 0 : md.ne, na = A == 0 ? md.ne : md.no;
    std::vector<float> upre((size_t)md.nc * V), upost((size_t)md.nc * V), lam((size_t)md.nc * V), w((size_t)na * V, 0.f);
    for (int c = 0; c < md.nc; ++c) {
        const size_t ic = (size_t)md.internal_of_abi[c];
        for (long long i = 0; i < V; ++i) {
            upre[ic * V + i] = (float)in[(size_t)c * V + i];
            upost[ic * V + i] = (float)in[(size_t)(md.nc + c) * V + i];
            lam[ic * V + i] = (float)in[(size_t)(2 * md.nc + c) * V + i];
        }
    }
    const adj::PullTable pt = adj::pull_table(md, A);
    std::vector<double> gacc((size_t)9 * V, 0.0), gq((size_t)V, 0.0);
    region(fac);
    region(upre);
    region(upost);
    region(lam);
    region(w);
    region(gacc);
    region(gq);
    region(pt.grp);
    region(pt.idx);
    const int fac_ofs = half ? FAC_HALF : FAC_FULL;
    const int pre_ofs = pre < 0 ? -1 : (pre ? FAC_HALF : FAC_FULL);
    for (long long c0 = 0; c0 < V; c0 += 4)
        adj::pull_cells(upre.data() + (size_t)a0 * V, upost.data() + (size_t)a0 * V, lam.data() + (size_t)a0 * V,
                        w.data(), fac.data(), dfac.data(), fac_ofs, pre_ofs, pt.grp.data(), (int)pt.grp.size() / 4,
                        pt.idx.data(), V, c0, gacc.data(), gq.data());
    std::vector<double> out((size_t)(2 * md.nc + 10) * V, 0.0);
    for (int c = 0; c < md.nc; ++c) {
        const int ic = md.internal_of_abi[c];
        for (long long i = 0; i < V; ++i) {
            if (ic >= a0 && ic < a0 + na) out[(size_t)c * V + i] = w[(size_t)(ic - a0) * V + i];
            out[(size_t)(md.nc + c) * V + i] = lam[(size_t)ic * V + i];
        }
    }
    std::copy(gacc.begin(), gacc.end(), out.begin() + (size_t)2 * md.nc * V);
    std::copy(gq.begin(), gq.end(), out.begin() + (size_t)(2 * md.nc + 9) * V);
    f = fopen(argv[12], "wb");
    fwrite(out.data(), 8, out.size(), f);
    fclose(f);
    return 0;
}
