// Host run of the TMA-staged substep kernel (test program): the kernel's own stage plan
// (stg::stage_box, stg::stage_bytes) and column work (stg::operand_offsets, stg::sweep_column,
// stg::finish_column), compiled for the host and driven CTA by CTA in the kernel's tile walk, over
// bounds-checked memory.  Each box of the plan is copied like the TMA unit copies it (a dense
// [E][z][y][x] box, coordinates outside the tensor read as zero, x aligned to 16 bytes); the
// consumers of every stage then run with their rotating accumulator window.  The program aborts
// on a box that leaves its region or its buffer, on an unaligned x coordinate, and on any read
// or write outside the ring, the state, the coupling constants or the factor planes.
//
// Compile with -DRTPN_SN=<order> -DRTPN_STX= -DRTPN_STY= -DRTPN_STZ= -DRTPN_SNB= -DRTPN_SEM= (a
// variant of stage_variants.h).
// usage: emulate_stage cls nx ny nz bc h dt half fp32|bf16 sms in.bin out.bin [adjsrc|adjsrc_alpha]
//   in.bin: float64 u [n_c][nz][ny][nx] (interface order), then sigma_a, sigma_s, q [nz][ny][nx]
//   out.bin: float64 u after the substep of class cls (tau = dt, or dt/2 with half = 1)
//   adjsrc: the adjoint's transposed coupling onto class cls instead (mode ADJ_SOURCES, FP32):
//     in.bin holds lam [n_c] and w [n_c] (interface order; w of the other class is used), then
//     the media; out.bin is lam after lam_B <- a lam_B + K w / h, with a = 1, or (adjsrc_alpha)
//     the class's factor at tau (u_0: its own)
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

static const char* g_lo[8];
static const char* g_hi[8];
static int g_nr = 0;
static void check_ptr(const void* p) {
    const char* c = (const char*)p;
    for (int i = 0; i < g_nr; ++i)
        if (c >= g_lo[i] && c < g_hi[i]) return;
    fprintf(stderr, "OUT OF BOUNDS access %p\n", p);
    std::abort();
}
static void fail(const char* what, long long v) {
    fprintf(stderr, "STAGE PLAN ERROR: %s (%lld)\n", what, v);
    std::abort();
}
#define RTPN_HOST_CHECK 1
#define RTPN_CHECK_PTR(p) check_ptr(p)
#include "stage_impl.cuh"

using namespace rtpn;
using namespace rtpn::stg;

constexpr int kN = RTPN_SN, kTX = RTPN_STX, kTY = RTPN_STY, kTZ = RTPN_STZ, kNB = RTPN_SNB, kEQ = RTPN_SEM;

// u: the target array (the state, or lam in mode ADJ_SOURCES), a full state; src: the source
// array with src_nc components (the state itself, or w of the source class in its local order)
template <int A, typename S>
void run(Args a, const float* fac, S* u, const S* src, int src_nc, const std::vector<float>& coef, int sms,
         int mode, bool use_alpha) {
    using L = Layout<kN, A, S, kTX, kTY, kTZ, kNB, kEQ>;
    constexpr int B = 1 - A, NST = kN + 2, NLA = (kN - A) / 2 + 1, CELLS = L::CELLS;
    constexpr int NJOB = 2 * L::NKIND + 2 * kTZ;
    if (!L::FITS) fail("variant does not fit this storage", 0);
    const long long V = a.V;
    const int cA0 = A == 0 ? 0 : class_size(kN, 0);
    const long long grid = a.tiles < sms ? a.tiles : sms;  // one persistent CTA per SM
    std::vector<unsigned char> ring((size_t)kNB * L::BUF);
    g_lo[3] = (const char*)ring.data();
    g_hi[3] = (const char*)(ring.data() + ring.size());
    // per consumer thread: three accumulator columns and the index of `prev` among them
    std::vector<float> win((size_t)2 * CELLS * 3 * NLA);
    std::vector<int> rot(2 * CELLS);
    for (long long cta = 0; cta < grid; ++cta) {
        std::fill(ring.begin(), ring.end(), 0);  // the kernel zeroes its ring once
        std::fill(rot.begin(), rot.end(), 0);
        const int my_tiles = (int)((a.tiles - 1 - cta) / grid) + 1;
        int offA = 0, offB = 0;
        unsigned tile = (unsigned)cta;
        TileGeo g{};
        for (int s = 0, i = 0; s < my_tiles * NST; ++s, i = (i == NST - 1) ? 0 : i + 1) {
            if (i == 0) {
                if (s > 0) tile += (unsigned)grid;
                g = tile_geo<kTX, kTY, kTZ, L::G>(a, tile);
                offA = offB = 0;
            }
            unsigned char* buf = ring.data() + (size_t)(s % kNB) * L::BUF;
            // ---- the producer's boxes, copied as the TMA unit copies them
            unsigned landed = 0;
            const StageRuns runs = stage_runs<kN, A>(i);
            for (int j = 0; j < NJOB; ++j) {
                const BoxJob bj = stage_box<kN, A, S, kTX, kTY, kTZ, kNB, kEQ>(a, g, i, runs, offA, offB, j);
                if (!bj.valid) continue;
                const int E = kEQ * (bj.emap + 1);
                int bx = kTX, by = kTY, bz = 1;
                if (!bj.target && bj.kind == MAP_YROW) by = 1, bz = kTZ;
                if (!bj.target && bj.kind == MAP_XGRP) bx = L::XW, by = L::RY, bz = kTZ;
                const int region_end = bj.target ? (bj.dst - L::TGTO) / L::REG * L::REG + L::REG + L::TGTO
                                                 : (bj.dst - L::SRCO) / L::REG * L::REG + L::REG + L::SRCO;
                const long long bytes = (long long)E * bx * by * bz * L::ES;
                if (bytes != (long long)E * L::UB) fail("box volume differs from E * U", bytes);
                if (bj.dst % 128 != 0) fail("box destination not 128-byte aligned", bj.dst);
                if (bj.dst + bytes > region_end || region_end > L::COEFO) fail("box leaves its region", bj.dst);
                if (((long long)bj.x * L::ES) % 16 != 0) fail("x coordinate not 16-byte aligned", bj.x);
                if (E < 1 || E > L::NL) fail("box length", E);
                const S* base = bj.target ? u : src;
                const int nc = bj.target ? class_size(kN, 0) + class_size(kN, 1) : src_nc;
                for (int ec = 0; ec < E; ++ec)
                    for (int ez = 0; ez < bz; ++ez)
                        for (int ey = 0; ey < by; ++ey)
                            for (int ex = 0; ex < bx; ++ex) {
                                const long long X = bj.x + ex, Y = bj.y + ey, Z = bj.z + ez, C = bj.c + ec;
                                S v{};
                                if (X >= 0 && X < a.nx && Y >= 0 && Y < a.ny && Z >= 0 && Z < a.nz && C >= 0 && C < nc) {
                                    const S* p = base + C * V + (Z * a.ny + Y) * a.nx + X;
                                    check_ptr(p);
                                    v = *p;
                                }
                                S* d = reinterpret_cast<S*>(buf + bj.dst) + (((ec * bz + ez) * by + ey) * bx + ex);
                                check_ptr(d);
                                *d = v;
                            }
                landed += (unsigned)bytes;
            }
            if (column_len(kN, i, B) > 0) {  // the coupling constants of column i (a plain bulk copy)
                const float* src = coef.data() + (size_t)i * (2 * L::NLC * CPAD);
                check_ptr(src);
                check_ptr(src + 2 * L::NLC * CPAD - 1);
                std::copy(src, src + 2 * L::NLC * CPAD, reinterpret_cast<float*>(buf + L::COEFO));
                landed += L::COEF_COL;
            }
            if (landed != stage_bytes<kN, A, S, kTX, kTY, kTZ, kNB, kEQ>(runs)) fail("expected bytes", landed);
            // ---- every consumer thread's column work
            for (int tid = 0; tid < 2 * CELLS; ++tid) {
                const int T = tid / CELLS, ctid = tid % CELLS;
                const int lx = ctid % kTX, ly = (ctid / kTX) % kTY, lz = ctid / (kTX * kTY);
                float* W = &win[(size_t)tid * 3 * NLA];
                if (i == 0) {
                    std::fill(W, W + 3 * NLA, 0.f);
                    rot[tid] = 0;
                }
                float(&prev)[NLA] = *reinterpret_cast<float(*)[NLA]>(W + rot[tid] * NLA);
                float(&cur)[NLA] = *reinterpret_cast<float(*)[NLA]>(W + ((rot[tid] + 1) % 3) * NLA);
                float(&next)[NLA] = *reinterpret_cast<float(*)[NLA]>(W + ((rot[tid] + 2) % 3) * NLA);
                const Operands op = operand_offsets<kN, A, S, kTX, kTY, kTZ, kNB, kEQ>(g, T, lx, ly, lz);
                if (column_len(kN, i, B) > 0) sweep_column<kN, A, S, kTX, kTY, kTZ, kNB, kEQ>(buf, op, T, i, prev, cur, next);
                if (i >= 1 && (T == 0 || i - 1 >= 1)) {
                    const int M = i - 1, q0 = first_l(M, A) / 2;
                    const bool active = lx < g.wx && ly < g.wy && lz < g.wz;
                    const long long cell = ((long long)(g.z0 + lz) * a.ny + (g.y0 + ly)) * a.nx + (g.x0 + lx);
                    float alpha = 0.f, beta = 0.f, al0 = 0.f, be0 = 0.f, ga0 = 0.f;
                    if (mode == ADJ_SOURCES && !use_alpha) alpha = al0 = 1.f;
                    if (active && (mode == FORWARD || use_alpha)) {
                        const int par = M & 1;
                        const int gx = ((par == 0) == (T == 0)) ? 0 : 1, gz = ((A + par) & 1) == 0 ? 0 : 1;
                        const int gc = gx + 2 * T + 4 * gz;
                        alpha = fac[(long long)(a.fac_ofs + 2 * gc) * V + cell];
                        beta = fac[(long long)(a.fac_ofs + 2 * gc + 1) * V + cell] * a.inv_h;
                        al0 = fac[(long long)FAC_U0 * V + cell];
                        be0 = fac[(long long)(FAC_U0 + 1) * V + cell] * a.inv_h;
                        ga0 = fac[(long long)(FAC_U0 + 2) * V + cell];
                    }
                    const int tgo = L::TGTO + T * L::TGT_T + lz * L::REG + (ly * kTX + lx) * L::ES;
                    S* tp = u + (long long)(cA0 + offA + T * column_len(kN, M, A) - q0) * V + cell;
                    if (mode == FORWARD)
                        finish_column<kN, A, S, kTX, kTY, kTZ, kNB, kEQ, FORWARD>(buf, tgo, M, T, tp, V, active, alpha,
                                                                                beta, al0, be0, ga0, a.inv_h, prev);
                    else
                        finish_column<kN, A, S, kTX, kTY, kTZ, kNB, kEQ, ADJ_SOURCES>(
                            buf, tgo, M, T, tp, V, active, alpha, beta, al0, be0, ga0, a.inv_h, prev);
                }
                std::fill(prev, prev + NLA, 0.f);
                rot[tid] = (rot[tid] + 1) % 3;
            }
            offB += ntypes(i) * column_len(kN, i, B);
            if (i >= 1) offA += ntypes(i - 1) * column_len(kN, i - 1, A);
        }
    }
}

int main(int argc, char** argv) {
    if (argc < 13) {
        fprintf(stderr, "usage\n");
        return 2;
    }
    const int A = atoi(argv[1]), nx = atoi(argv[2]), ny = atoi(argv[3]), nz = atoi(argv[4]), bc = atoi(argv[5]);
    const double h = atof(argv[6]), dt = atof(argv[7]);
    const int half = atoi(argv[8]);
    const std::string prec = argv[9];
    const int sms = atoi(argv[10]);
    const char* inf = argv[11];
    const char* outf = argv[12];
    const std::string mode_s = argc > 13 ? argv[13] : "fwd";
    const int mode = mode_s == "fwd" ? FORWARD : ADJ_SOURCES;
    const bool use_alpha = mode_s == "adjsrc_alpha";
    if (mode == ADJ_SOURCES && prec != "fp32") {
        fprintf(stderr, "the transposed coupling runs on FP32 arrays\n");
        return 2;
    }
    const int N = kN;
    Model md = build_model(N);
    const long long V = (long long)nx * ny * nz;
    const int narr = mode == FORWARD ? 1 : 2;  // u, or lam and w
    std::vector<double> in((size_t)(narr * md.nc + 3) * V);
    FILE* f = fopen(inf, "rb");
    if (!f || fread(in.data(), 8, in.size(), f) != in.size()) {
        fprintf(stderr, "bad input\n");
        return 4;
    }
    fclose(f);
    const double* sa = in.data() + (size_t)narr * md.nc * V;
    const double* ss = sa + V;
    const double* q = ss + V;
    // factor planes by the rule of rtpn_set_media (mean of sigma over the cells adjacent to a
    // sub-grid point; alpha = exp(-c tau), beta = tau E(-c tau)), FP32
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
    std::vector<int> col;
    std::vector<float> tab[2];
    if (!coupling_tables(md, 1.0, 1.0, tab, &col)) {
        fprintf(stderr, "coupling tables\n");
        return 3;
    }
    Args a{};
    a.V = V;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.bc = bc;
    a.fac_ofs = half ? FAC_HALF : FAC_FULL;
    a.inv_h = (float)(1.0 / h);
    a.ntx = (nx + kTX - 1) / kTX;
    a.nty = (ny + kTY - 1) / kTY;
    a.ntz = (nz + kTZ - 1) / kTZ;
    a.tiles = (long long)a.ntx * a.nty * a.ntz;
    {
        const double side = std::sqrt((double)sms / a.ntx);
        const int kz = (int)(side + 0.5);
        a.kz = kz < 1 ? 1 : (kz > a.ntz ? a.ntz : kz);
    }
    a.src_c0 = A == 1 ? 0 : md.ne;  // the source class is the other one
    a.nc = md.nc;
    // mode ADJ_SOURCES: w of the other class, in its local order, is the source array
    const int aw0 = A == 1 ? 0 : md.ne, nw = A == 1 ? md.ne : md.no;
    std::vector<float> wloc;
    if (mode == ADJ_SOURCES) {
        wloc.resize((size_t)nw * V);
        const double* w = in.data() + (size_t)md.nc * V;
        for (int c = 0; c < md.nc; ++c) {
            const int ic = md.internal_of_abi[c];
            if (ic < aw0 || ic >= aw0 + nw) continue;
            for (long long i = 0; i < V; ++i) wloc[(size_t)(ic - aw0) * V + i] = (float)w[(size_t)c * V + i];
        }
        a.src_c0 = 0;
        a.nc = nw;
        g_lo[4] = (const char*)wloc.data();
        g_hi[4] = (const char*)(wloc.data() + wloc.size());
    }
    g_lo[0] = (const char*)fac.data();
    g_hi[0] = (const char*)(fac.data() + fac.size());
    g_lo[1] = (const char*)tab[A].data();
    g_hi[1] = (const char*)(tab[A].data() + tab[A].size());
    std::vector<double> out((size_t)md.nc * V);
    auto go = [&](auto tag) {
        using S = decltype(tag);
        std::vector<S> u((size_t)md.nc * V);
        for (int c = 0; c < md.nc; ++c)
            for (long long i = 0; i < V; ++i) {
                const double v = in[(size_t)c * V + i];
                if constexpr (sizeof(S) == 4)
                    u[(size_t)md.internal_of_abi[c] * V + i] = (float)v;
                else
                    u[(size_t)md.internal_of_abi[c] * V + i] = __float2bfloat16_rn((float)v);
            }
        g_lo[2] = (const char*)u.data();
        g_hi[2] = (const char*)(u.data() + u.size());
        g_nr = mode == FORWARD ? 4 : 5;
        const S* src = u.data();
        int src_nc = md.nc;
        if constexpr (sizeof(S) == 4) {
            if (mode == ADJ_SOURCES) {
                src = wloc.data();
                src_nc = nw;
            }
        }
        if (A == 0)
            run<0, S>(a, fac.data(), u.data(), src, src_nc, tab[0], sms, mode, use_alpha);
        else
            run<1, S>(a, fac.data(), u.data(), src, src_nc, tab[1], sms, mode, use_alpha);
        for (int c = 0; c < md.nc; ++c)
            for (long long i = 0; i < V; ++i) {
                const S v = u[(size_t)md.internal_of_abi[c] * V + i];
                if constexpr (sizeof(S) == 4)
                    out[(size_t)c * V + i] = v;
                else
                    out[(size_t)c * V + i] = __bfloat162float(v);
            }
    };
    if (prec == "fp32")
        go(float{});
    else
        go(__nv_bfloat16{});
    f = fopen(outf, "wb");
    fwrite(out.data(), 8, out.size(), f);
    fclose(f);
    return 0;
}
