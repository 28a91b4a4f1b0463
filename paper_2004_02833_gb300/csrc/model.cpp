// Closed-form coupling coefficients of the real P_N system (Eq. 3) and the staggered placement
// (Section 2.1), generated on the host in FP64.
//
// Basis (no Condon-Shortley phase): p_l^m(mu) = sqrt(2 pi) N_l^m P_l^m(mu) is orthonormal on
// [-1, 1] for fixed m; the angular factors are 1/sqrt(2 pi) (m = 0), cos(m phi)/sqrt(pi) and
// sin(m phi)/sqrt(pi).  Every entry M_d[a][b] = int Omega_d Y_a Y_b dOmega factors into a mu
// integral and a phi integral.
//
// mu integrals (the Legendre ladder relations, P_l^m = (1-mu^2)^{m/2} d^m P_l / dmu^m):
//   mu P_l^m              = ((l-m+1) P_{l+1}^m + (l+m) P_{l-1}^m) / (2l+1)
//   sqrt(1-mu^2) P_l^m    = (P_{l+1}^{m+1} - P_{l-1}^{m+1}) / (2l+1)
// which after normalisation give
//   int mu p_l^m p_{l+1}^m            = sqrt(((l+1)^2 - m^2) / ((2l+1)(2l+3)))
//   int sqrt(1-mu^2) p_l^m p_{l+1}^{m+1} =  sqrt((l+m+1)(l+m+2) / ((2l+1)(2l+3)))
//   int sqrt(1-mu^2) p_l^m p_{l-1}^{m+1} = -sqrt((l-m)(l-m-1) / ((2l-1)(2l+1)))
// phi integrals for m' = m + 1 (Omega_x carries cos phi, Omega_y sin phi):
//   cos phi:  m = 0 -> cos: 1/sqrt(2);  cos m -> cos m+1: 1/2;  sin m -> sin m+1: 1/2
//   sin phi:  m = 0 -> sin: 1/sqrt(2);  cos m -> sin m+1: 1/2;  sin m -> cos m+1: -1/2
// and zero for every other pair.  Mz keeps m and the type.
//
// Slots: a real basis function is even or odd under x -> -x (phi -> pi - phi), y -> -y
// (phi -> -phi) and z -> -z (mu -> -mu): cos type has parities ((-1)^m, +1), sin type
// (-(-1)^m, -1) in x and y, and (-1)^(l+m) in z.  Omega_d is odd in d only, so a nonzero of M_d
// joins functions that differ in the d parity alone; slot 1 = even parity puts u_0 on G111 and
// makes every d-derivative switch slot d, as Section 2.1 requires.
#include "model.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace rtpn {

namespace {

double mz_coef(int l, int M) {  // between (l, M) and (l+1, M)
    return std::sqrt(double((l + 1) * (l + 1) - M * M) / double((2 * l + 1) * (2 * l + 3)));
}

double ladder_up(int l, int M) {  // sqrt(1-mu^2): (l, M) with (l+1, M+1)
    return std::sqrt(double((l + M + 1) * (l + M + 2)) / double((2 * l + 1) * (2 * l + 3)));
}

double ladder_down(int l, int M) {  // sqrt(1-mu^2): (l, M) with (l-1, M+1)
    return -std::sqrt(double((l - M) * (l - M - 1)) / double((2 * l - 1) * (2 * l + 1)));
}

void add(Model& md, int a, int b, int axis, double v) {
    md.nz.push_back({a, b, axis, v});
    md.nz.push_back({b, a, axis, v});
}

}  // namespace

Model build_model(int N) {
    if (N < 0 || N > 63) throw std::invalid_argument("N out of range");
    Model md;
    md.N = N;
    md.nc = (N + 1) * (N + 1);
    md.comp.resize(md.nc);
    for (int l = 0; l <= N; ++l) {
        for (int m = -l; m <= l; ++m) {
            Component c;
            c.l = l;
            c.M = std::abs(m);
            c.t = m < 0 ? 1 : 0;
            c.m = m;
            c.abi = l * l + l + m;
            const int sgnM = (c.M % 2 == 0) ? 1 : -1;
            const int px = c.t == 0 ? sgnM : -sgnM;
            const int py = c.t == 0 ? 1 : -1;
            const int pz = ((l + c.M) % 2 == 0) ? 1 : -1;
            c.slot[0] = px == 1 ? 1 : 2;
            c.slot[1] = py == 1 ? 1 : 2;
            c.slot[2] = pz == 1 ? 1 : 2;
            c.cls = l % 2;
            md.comp[c.abi] = c;
        }
    }
    // internal order: class, M, t, l
    for (int cls = 0; cls < 2; ++cls)
        for (int M = 0; M <= N; ++M)
            for (int t = 0; t < (M == 0 ? 1 : 2); ++t)
                for (int l = M; l <= N; ++l)
                    if (l % 2 == cls) md.abi_of_internal.push_back(abi_index(l, M, t));
    md.internal_of_abi.assign(md.nc, -1);
    for (int i = 0; i < md.nc; ++i) md.internal_of_abi[md.abi_of_internal[i]] = i;
    md.ne = 0;
    for (const auto& c : md.comp) md.ne += (c.cls == 0);
    md.no = md.nc - md.ne;

    const double r2 = 1.0 / std::sqrt(2.0);
    for (int l = 0; l <= N; ++l) {
        for (int M = 0; M <= l; ++M) {
            for (int t = 0; t < (M == 0 ? 1 : 2); ++t) {
                const int a = abi_index(l, M, t);
                if (l + 1 <= N) add(md, a, abi_index(l + 1, M, t), 2, mz_coef(l, M));
                // couplings to |m| = M + 1
                for (int dl = -1; dl <= 1; dl += 2) {
                    const int lp = l + dl;
                    if (lp < M + 1 || lp > N) continue;
                    const double I = dl > 0 ? ladder_up(l, M) : ladder_down(l, M);
                    if (I == 0.0) continue;
                    const double Jx = M == 0 ? r2 : 0.5;
                    add(md, a, abi_index(lp, M + 1, t), 0, I * Jx);
                    if (t == 0) {
                        add(md, a, abi_index(lp, M + 1, 1), 1, I * (M == 0 ? r2 : 0.5));
                    } else {
                        add(md, a, abi_index(lp, M + 1, 0), 1, -0.5 * I);
                    }
                }
            }
        }
    }
    std::sort(md.nz.begin(), md.nz.end(), [](const Coupling& x, const Coupling& y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.axis != y.axis) return x.axis < y.axis;
        return x.b < y.b;
    });
    return md;
}

}  // namespace rtpn
