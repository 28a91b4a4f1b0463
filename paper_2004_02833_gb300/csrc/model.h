// Host-side model of the P_N component set: interface order, internal order, sub-grid slots and
// the sparse coupling entries of Mx, My, Mz (Eq. 3), generated in FP64 from closed forms.
#pragma once

#include <vector>

namespace rtpn {

struct Component {
    int l;        // moment order
    int M;        // |m|
    int t;        // 0: cos type (or m = 0), 1: sin type
    int m;        // signed m (m > 0 cos, m < 0 sin)
    int abi;      // interface index l*l + l + m
    int slot[3];  // sub-grid slot along x, y, z (1 or 2)
    int cls;      // 0: even grid (even l), 1: odd grid (odd l)
};

struct Coupling {
    int a, b;     // interface indices (row, column)
    int axis;     // 0 x, 1 y, 2 z
    double v;     // M_axis[a][b]
};

struct Model {
    int N = 0, nc = 0, ne = 0, no = 0;
    std::vector<Component> comp;            // by interface index
    std::vector<int> internal_of_abi;       // interface -> internal index
    std::vector<int> abi_of_internal;       // internal -> interface index
    std::vector<Coupling> nz;               // every nonzero of Mx, My, Mz (both triangles)
};

// Interface index of (l, M, t).
inline int abi_index(int l, int M, int t) { return l * l + l + (t == 0 ? M : -M); }

// Builds the model for order N (0 <= N <= 63).  Internal order: class (even first), then M
// ascending, then type (cos before sin), then l ascending; each (class, M, t) run shares one
// sub-grid.
Model build_model(int N);

// Slot code g = (gx-1) + 2 (gy-1) + 4 (gz-1) in 0..7.
inline int slot_code(const int s[3]) { return (s[0] - 1) + 2 * (s[1] - 1) + 4 * (s[2] - 1); }

}  // namespace rtpn
