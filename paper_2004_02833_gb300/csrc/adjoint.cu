// Discrete adjoint of the staggered P_N step: gradients of a detector functional with respect to the
// per-cell media.
//
// A substep on class A (Eq. 5 rearranged) is
//     u_A' = alpha_A u_A + beta_A r_A,   r_A = q_A - sum_d M_d^{AB} D_d u_B,   u_B' = u_B,
// with alpha = exp(-c tau), beta = tau E(-c tau) at each component's staggered point.  For
// J = sum_cells w u_0 after k steps, the pull-back of lam' = dJ/du' through that substep is
//     lam_A = alpha_A lam'_A,   lam_B = lam'_B - sum_a K_{ab}^T (beta_a lam'_a),
// where K^T is the transposed staggered stencil (a forward difference becomes a negated backward
// difference with the same boundary rule), and the media receive
//     dJ/dc_a += lam'_a (dalpha/dc u_a + dbeta/dc r_a),   dJ/dq += beta_0 lam'_0,
// with dalpha/dc = -tau alpha and dbeta/dc = -tau^2 E'(-c tau), E'(x) = (e^x (x - 1) + 1) / x^2.
// dJ/dc at the staggered points is spread back to the cells by the transpose of the point mean.
//
// With the generic kernels (FP64, the parity path) the forward is the literal Strang step (odd half,
// even full, odd half), so that the adjoint is the exact transpose of the computed scheme.  States
// are checkpointed every `ckpt` steps; each segment is recomputed forward (with the active step
// kernel) keeping every pre-substep state, then swept backward with k_adj_targets and
// k_adj_sources.  FP32 storage on the staged kernel runs the merged form of the step with
// out-of-place segment states and a cell-by-cell pull-back (adjoint_staged).  Gradient accumulators
// are FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "pull_impl.cuh"
#include "rtpn_internal.h"

namespace rtpn {
namespace {

template <typename S, typename F>
__device__ __forceinline__ F ldv(const S* p) { return static_cast<F>(*p); }
template <>
__device__ __forceinline__ float ldv<__nv_bfloat16, float>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}

__device__ __forceinline__ bool nb_cell(const Geom& g, int x, int y, int z, int axis, int dir, long long* idx) {
    int c[3] = {x, y, z};
    const int n[3] = {g.nx, g.ny, g.nz};
    int v = c[axis] + dir;
    if (v < 0 || v >= n[axis]) {
        if (g.bc != RTPN_BC_PERIODIC) return false;
        v = v < 0 ? v + n[axis] : v - n[axis];
    }
    c[axis] = v;
    *idx = ((long long)c[2] * g.ny + c[1]) * g.nx + c[0];
    return true;
}

using adj::DFAC_PLANES;

template <typename F>
__global__ void k_adj_factors(const double* __restrict__ sa, const double* __restrict__ ss, F* __restrict__ dfac,
                              Geom g, double dt) {
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell < g.V) adj::factor_derivatives<F>(sa, ss, dfac, g, dt, cell);
}

// Targets of class A: forward residual on the pre-substep state, media gradients, w = beta lam,
// lam_A <- alpha lam_A.  gacc[9][V]: dJ/dc per slot code (0..7) and for u_0 (8); gq[V]: dJ/dq.
template <typename S, typename F>
__global__ void k_adj_targets(const S* __restrict__ u, F* __restrict__ lam, F* __restrict__ w,
                              const F* __restrict__ fac, const F* __restrict__ dfac, PartnerTable<F> tab,
                              Geom g, int fac_ofs, const double* __restrict__ q, double* __restrict__ gacc,
                              double* __restrict__ gq) {
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= g.V) return;
    const int x = (int)(cell % g.nx), y = (int)((cell / g.nx) % g.ny), z = (int)(cell / ((long long)g.nx * g.ny));
    long long nb[6];
    bool ok[6];
    for (int code = 0; code < 6; ++code) {
        ok[code] = nb_cell(g, x, y, z, code >> 1, (code & 1) ? 1 : -1, &nb[code]);
        if (!ok[code]) nb[code] = cell;
    }
    double gs[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double gqa = 0.0;
    for (int t = 0; t < tab.na; ++t) {
        F r = F(0);
        for (int p = tab.row[t]; p < tab.row[t + 1]; ++p) {
            const S* ub = u + (long long)tab.src[p] * g.V;
            const int code = tab.code[p];
            const F centre = ldv<S, F>(ub + cell);
            const F other = ok[code] ? ldv<S, F>(ub + nb[code]) : F(0);
            r -= tab.coef[p] * (other - centre);
        }
        const int fp = tab.fplane[t];
        const long long ai = (long long)(tab.a0 + t) * g.V + cell;
        const F ua = ldv<S, F>(u + ai);
        const F la = lam[ai];
        F al, be, da, db;
        int slot;
        if (fp == FAC_U0) {
            al = fac[(long long)FAC_U0 * g.V + cell];
            be = fac[(long long)(FAC_U0 + 1) * g.V + cell];
            r += (F)q[cell];  // the source enters the u_0 residual
            da = dfac[(long long)32 * g.V + cell];
            db = dfac[(long long)33 * g.V + cell];
            slot = 8;
            gqa += (double)be * (double)la;
        } else {
            al = fac[(long long)(fp + fac_ofs) * g.V + cell];
            be = fac[(long long)(fp + fac_ofs + 1) * g.V + cell];
            da = dfac[(long long)(fp + fac_ofs) * g.V + cell];
            db = dfac[(long long)(fp + fac_ofs + 1) * g.V + cell];
            slot = fp / 2;
        }
        gs[slot] += (double)la * ((double)da * (double)ua + (double)db * (double)r);
        w[(long long)t * g.V + cell] = be * la;
        lam[ai] = al * la;
    }
    for (int s = 0; s < 9; ++s)
        if (gs[s] != 0.0) gacc[(long long)s * g.V + cell] += gs[s];
    if (gqa != 0.0) gq[cell] += gqa;
}

// Sources of class B: lam_b -= sum_a coefT * (w_a(neighbour) - w_a(cell)).
template <typename F>
__global__ void k_adj_sources(F* __restrict__ lam, const F* __restrict__ w, PartnerTable<F> tabT, int w_a0,
                              Geom g) {
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= g.V) return;
    const int x = (int)(cell % g.nx), y = (int)((cell / g.nx) % g.ny), z = (int)(cell / ((long long)g.nx * g.ny));
    long long nb[6];
    bool ok[6];
    for (int code = 0; code < 6; ++code) {
        ok[code] = nb_cell(g, x, y, z, code >> 1, (code & 1) ? 1 : -1, &nb[code]);
        if (!ok[code]) nb[code] = cell;
    }
    for (int t = 0; t < tabT.na; ++t) {
        F acc = F(0);
        for (int p = tabT.row[t]; p < tabT.row[t + 1]; ++p) {
            const F* wa = w + (long long)(tabT.src[p] - w_a0) * g.V;
            const int code = tabT.code[p];
            const F other = ok[code] ? wa[nb[code]] : F(0);
            acc += tabT.coef[p] * (other - wa[cell]);
        }
        lam[(long long)(tabT.a0 + t) * g.V + cell] -= acc;
    }
}

// The pull-back through a pass on class A from its stored pre- and post-pass states, four cells per
// thread (adj::pull_cells; V % 4 == 0, so every plane starts 16-byte aligned).
__global__ void __launch_bounds__(256) k_adj_pull(const float* __restrict__ upre, const float* __restrict__ upost,
                                                  float* __restrict__ lam, float* __restrict__ w,
                                                  const float* __restrict__ fac, const float* __restrict__ dfac,
                                                  int fac_ofs, int pre_ofs, const int* __restrict__ grp, int ngroups,
                                                  const int* __restrict__ idx, long long V,
                                                  double* __restrict__ gacc, double* __restrict__ gq) {
    const long long c0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (c0 < V)
        adj::pull_cells(upre, upost, lam, w, fac, dfac, fac_ofs, pre_ofs, grp, ngroups, idx, V, c0, gacc, gq);
}

// Transpose of the point mean: every staggered point spreads its dJ/dc over its adjacent cells.
__global__ void k_adj_media(const double* __restrict__ gacc, Geom g, double* __restrict__ g_sa,
                            double* __restrict__ g_ss) {
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= g.V) return;
    const int x = (int)(cell % g.nx), y = (int)((cell / g.nx) % g.ny), z = (int)(cell / ((long long)g.nx * g.ny));
    const int n[3] = {g.nx, g.ny, g.nz};
    double tot = 0.0;
    for (int code = 0; code < 8; ++code) {
        const int gd[3] = {code & 1, (code >> 1) & 1, (code >> 2) & 1};
        // points i = cell - delta (delta in {0,1} on the 2-slot axes) whose cell set holds this cell
        for (int dz = 0; dz <= gd[2]; ++dz)
            for (int dy = 0; dy <= gd[1]; ++dy)
                for (int dx = 0; dx <= gd[0]; ++dx) {
                    int p[3] = {x - dx, y - dy, z - dz};
                    bool inside = true;
                    for (int d = 0; d < 3; ++d)
                        if (p[d] < 0) {
                            if (g.bc == RTPN_BC_PERIODIC)
                                p[d] += n[d];
                            else
                                inside = false;
                        }
                    if (!inside) continue;
                    // the point's count of in-domain adjacent cells
                    int cnt = 1;
                    for (int d = 0; d < 3; ++d)
                        if (gd[d]) cnt *= (g.bc == RTPN_BC_PERIODIC || p[d] + 1 < n[d]) ? 2 : 1;
                    const long long pi = ((long long)p[2] * g.ny + p[1]) * g.nx + p[0];
                    tot += gacc[(long long)code * g.V + pi] / cnt;
                }
    }
    g_ss[cell] = tot;
    g_sa[cell] = tot + gacc[(long long)8 * g.V + cell];
}

template <typename S>
__global__ void k_dot_u0(const S* __restrict__ u0, const double* __restrict__ w, long long n,
                         double* __restrict__ partial) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)ldv<S, float>(u0 + i) * w[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i];
        partial[blockIdx.x] = s;
    }
}
template <>
__global__ void k_dot_u0<double>(const double* __restrict__ u0, const double* __restrict__ w, long long n,
                                 double* __restrict__ partial) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += u0[i] * w[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i];
        partial[blockIdx.x] = s;
    }
}

template <typename A, typename B>
__global__ void k_copy_cast(const A* __restrict__ in, B* __restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}

unsigned blocks_for(long long V, int threads = 256) { return (unsigned)((V + threads - 1) / threads); }

// out = sum of partial[0 .. count) in a fixed order (one block)
__global__ void k_partials_total(const double* __restrict__ partial, int count, double* __restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i];
        *out = s;
    }
}

}  // namespace

// Transposed partner table of class B targets (sources = class A, the w planes), host side.
HostTable transposed_table(const Model& md, int clsB, const Geom& g) {
    HostTable t;
    t.a0 = clsB == 0 ? 0 : md.ne;
    t.na = clsB == 0 ? md.ne : md.no;
    std::vector<std::vector<int>> col(md.nc);  // entries with column b
    for (size_t q = 0; q < md.nz.size(); ++q) col[md.nz[q].b].push_back((int)q);
    t.row.push_back(0);
    for (int i = t.a0; i < t.a0 + t.na; ++i) {
        const int b = md.abi_of_internal[i];
        for (int q : col[b]) {
            const Coupling& e = md.nz[q];  // M[a][b], target a of the forward substep
            const Component& ca = md.comp[e.a];
            // forward: slot 2 reads b at i, i+1 -> transpose reads w_a at j-1, j with + M/h;
            //          slot 1 reads b at i-1, i -> transpose reads w_a at j, j+1 with - M/h.
            const bool a_upper = ca.slot[e.axis] == 2;
            t.src.push_back(md.internal_of_abi[e.a]);
            t.code.push_back(e.axis * 2 + (a_upper ? 0 : 1));
            t.coef.push_back((a_upper ? 1.0 : -1.0) * e.v / axis_h(g, e.axis));
        }
        t.row.push_back((int)t.src.size());
        t.fplane.push_back(0);
    }
    return t;
}

}  // namespace rtpn

using namespace rtpn;

namespace {

int afail(rtpn_ctx* ctx, int code, const std::string& msg) {
    ctx->err = msg;
    return code;
}

template <typename F>
struct DevTable {
    int* ints = nullptr;
    F* coef = nullptr;
    PartnerTable<F> tab{};
    ~DevTable() {
        if (ints) cudaFree(ints);
        if (coef) cudaFree(coef);
    }
    bool upload(const HostTable& h) {
        const size_t ni = h.row.size() + h.src.size() + h.code.size() + h.fplane.size();
        if (cudaMalloc(&ints, ni * sizeof(int)) != cudaSuccess) return false;
        if (cudaMalloc(&coef, (h.coef.size() + 1) * sizeof(F)) != cudaSuccess) return false;
        std::vector<int> all;
        all.insert(all.end(), h.row.begin(), h.row.end());
        all.insert(all.end(), h.src.begin(), h.src.end());
        all.insert(all.end(), h.code.begin(), h.code.end());
        all.insert(all.end(), h.fplane.begin(), h.fplane.end());
        std::vector<F> cf(h.coef.begin(), h.coef.end());
        cudaMemcpy(ints, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(coef, cf.data(), cf.size() * sizeof(F), cudaMemcpyHostToDevice);
        tab.row = ints;
        tab.src = ints + h.row.size();
        tab.code = ints + h.row.size() + h.src.size();
        tab.fplane = ints + h.row.size() + h.src.size() + h.code.size();
        tab.coef = coef;
        tab.a0 = h.a0;
        tab.na = h.na;
        return true;
    }
};

// RAII device buffer
struct Buf {
    void* p = nullptr;
    ~Buf() {
        if (p) cudaFree(p);
    }
    bool alloc(size_t n) { return cudaMalloc(&p, n) == cudaSuccess; }
};

template <typename S, typename F>
int adjoint_impl(rtpn_ctx* ctx, const double* w_dev, int k, int ckpt, double* gsa, double* gss, double* gq_out,
                 double* J) {
    const Geom& g = ctx->g;
    const long long V = g.V;
    const int nc = ctx->md.nc;
    const size_t state = (size_t)nc * V * sizeof(S);
    cudaStream_t st = ctx->stream;
    const int nseg = (k + ckpt - 1) / ckpt;
    const int npass = 3 * ckpt;  // pre-substep states kept per segment

    Buf ck, seg, lam, wbuf, dfac, gacc, gqb, part, media;
    if (!ck.alloc(state * nseg) || !seg.alloc(state * npass) || !lam.alloc((size_t)nc * V * sizeof(F)) ||
        !wbuf.alloc((size_t)std::max(ctx->md.ne, ctx->md.no) * V * sizeof(F)) ||
        !dfac.alloc((size_t)DFAC_PLANES * V * sizeof(F)) || !gacc.alloc((size_t)9 * V * sizeof(double)) ||
        !gqb.alloc((size_t)V * sizeof(double)) || !part.alloc(1024 * sizeof(double)))
        return afail(ctx, RTPN_ENOMEM, "adjoint: device memory for checkpoints and segment states");
    DevTable<F> tt[2];
    const PartnerTable<F>* tf = nullptr;
    if constexpr (sizeof(F) == 8)
        tf = reinterpret_cast<const PartnerTable<F>*>(ctx->tab64);
    else
        tf = reinterpret_cast<const PartnerTable<F>*>(ctx->tab32);
    for (int c = 0; c < 2; ++c)
        if (!tt[c].upload(transposed_table(ctx->md, c, g)))
            return afail(ctx, RTPN_ENOMEM, "adjoint: tables");
    k_adj_factors<F><<<blocks_for(V), 256, 0, st>>>(ctx->media, ctx->media + V, (F*)dfac.p, g, ctx->dt);

    // ---- forward with checkpoints (literal Strang steps)
    S* u = (S*)ctx->u;
    auto step3 = [&](cudaStream_t s, S* keep) -> int {
        const int cls[3] = {1, 0, 1}, ofs[3] = {FAC_HALF, FAC_FULL, FAC_HALF};
        for (int p = 0; p < 3; ++p) {
            if (keep) cudaMemcpyAsync((char*)keep + (size_t)p * state, u, state, cudaMemcpyDeviceToDevice, s);
            int rc = rtpn_substep(ctx, cls[p], ofs[p] == FAC_HALF);
            if (rc) return rc;
        }
        return RTPN_OK;
    };
    for (int s = 0; s < k; ++s) {
        if (s % ckpt == 0)
            cudaMemcpyAsync((char*)ck.p + (size_t)(s / ckpt) * state, u, state, cudaMemcpyDeviceToDevice, st);
        int rc = step3(st, nullptr);
        if (rc) return rc;
    }
    // J = sum w u_0 (u_0 is internal component 0)
    k_dot_u0<S><<<1024, 256, 0, st>>>(u, w_dev, V, (double*)part.p);
    launch_sum<double>((const double*)part.p, 1024, ctx->partial, 1, ctx->partial + SUM_BLOCKS, st);
    cudaMemcpyAsync(J, ctx->partial + SUM_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, st);

    // ---- backward
    cudaMemsetAsync(lam.p, 0, (size_t)nc * V * sizeof(F), st);
    k_copy_cast<double, F><<<1024, 256, 0, st>>>(w_dev, (F*)lam.p, V);  // lam_0 = w
    cudaMemsetAsync(gacc.p, 0, (size_t)9 * V * sizeof(double), st);
    cudaMemsetAsync(gqb.p, 0, (size_t)V * sizeof(double), st);
    // keep the final state to restore it afterwards
    Buf fin;
    if (!fin.alloc(state)) return afail(ctx, RTPN_ENOMEM, "adjoint: final state");
    cudaMemcpyAsync(fin.p, u, state, cudaMemcpyDeviceToDevice, st);
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int s0 = sg * ckpt, s1 = std::min(k, s0 + ckpt);
        cudaMemcpyAsync(u, (char*)ck.p + (size_t)sg * state, state, cudaMemcpyDeviceToDevice, st);
        for (int s = s0; s < s1; ++s) {
            int rc = step3(st, (S*)((char*)seg.p + (size_t)(s - s0) * 3 * state));
            if (rc) return rc;
        }
        for (int p = 3 * (s1 - s0) - 1; p >= 0; --p) {
            const int cls = (p % 3 == 1) ? 0 : 1;
            const int ofs = (p % 3 == 1) ? FAC_FULL : FAC_HALF;
            const S* pre = (const S*)((char*)seg.p + (size_t)p * state);
            k_adj_targets<S, F><<<blocks_for(V, 128), 128, 0, st>>>(pre, (F*)lam.p, (F*)wbuf.p, (const F*)ctx->fac,
                                                               (const F*)dfac.p, tf[cls], g, ofs, ctx->media + 2 * V,
                                                               (double*)gacc.p, (double*)gqb.p);
            k_adj_sources<F><<<blocks_for(V, 128), 128, 0, st>>>((F*)lam.p, (const F*)wbuf.p, tt[1 - cls].tab,
                                                            tf[cls].a0, g);
        }
    }
    cudaMemcpyAsync(u, fin.p, state, cudaMemcpyDeviceToDevice, st);
    k_adj_media<<<blocks_for(V), 256, 0, st>>>((const double*)gacc.p, g, gsa, gss);
    cudaMemcpyAsync(gq_out, gqb.p, (size_t)V * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return afail(ctx, RTPN_ECUDA, std::string("adjoint: ") + cudaGetErrorString(e));
    ctx->steps_done += k;
    return RTPN_OK;
}

using adj::PullTable;
using adj::pull_table;

// FP32 storage on the staged kernel.  The k steps run as segments of ckpt whole Strang steps, each in
// the merged form of the step (odd half pass; even and odd full passes; even full pass; odd half
// pass): two odd half passes with no even pass between them are one odd full pass in exact
// arithmetic (alpha_h^2 = alpha, beta_h (1 + alpha_h) = beta), so this is the literal schedule up
// to rounding.  The passes of a segment write out of place: pass j writes its class into X[j/2 + 1],
// its old targets come from X[j/2] and its sources from X[(j+1)/2], with X[0] the segment's
// checkpoint.  Every pass's pre- and post-pass values then stay in memory without copies, and the
// backward sweep recovers each pass's residual cell by cell (k_adj_pull) instead of re-running its
// stencil; the transposed coupling runs on the staged kernel (mode ADJ_SOURCES) and also applies
// the pulled-back class's pending lam <- alpha lam.  The last segment's states are still in place
// after the forward, so only the earlier ones are recomputed.
int adjoint_staged(rtpn_ctx* ctx, const double* w_dev, int k, int ckpt, double* gsa, double* gss, double* gq_out,
                   double* J) {
    const Geom& g = ctx->g;
    const long long V = g.V;
    const int nc = ctx->md.nc, ne = ctx->md.ne, no = ctx->md.no;
    const size_t state = (size_t)nc * V * sizeof(float);
    cudaStream_t st = ctx->stream;
    const int nseg = (k + ckpt - 1) / ckpt;
    const int nring = std::min(k, ckpt) + 1;  // X[1] .. X[m + 1] of the longest segment
    const size_t mapb = stage_maps_bytes(ctx);
    if (V % 4 != 0 || mapb == 0) return afail(ctx, RTPN_EUNSUPPORTED, "adjoint: staged kernel layout");
    // the pull-back's component groups of both classes, for one device array
    PullTable pt[2] = {pull_table(ctx->md, 0), pull_table(ctx->md, 1)};
    std::vector<int> all;
    size_t at[2][2];
    for (int c = 0; c < 2; ++c) {
        at[c][0] = all.size();
        all.insert(all.end(), pt[c].grp.begin(), pt[c].grp.end());
        at[c][1] = all.size();
        all.insert(all.end(), pt[c].idx.begin(), pt[c].idx.end());
    }
    // work buffers carved from the context's workspace, which is kept between calls
    enum { CK, RING, LAM, WB, DFAC, GACC, GQ, PART, MAPS, TABS, NBUF };
    const size_t need[NBUF] = {state * std::max(nseg, 1), state * nring, state,
                               (size_t)std::max(ne, no) * V * sizeof(float),
                               (size_t)DFAC_PLANES * V * sizeof(float), (size_t)9 * V * sizeof(double),
                               (size_t)V * sizeof(double), 1024 * sizeof(double), (size_t)(nseg + nring) * mapb,
                               all.size() * sizeof(int)};
    size_t off[NBUF], total = 0;
    for (int k = 0; k < NBUF; ++k) {
        off[k] = total;
        total += (need[k] + 255) / 256 * 256;
    }
    if (ctx->adj_ws_bytes < total) {
        if (ctx->adj_ws) cudaFree(ctx->adj_ws);
        ctx->adj_ws = nullptr;
        ctx->adj_ws_bytes = 0;
        if (cudaMalloc(&ctx->adj_ws, total) != cudaSuccess) {
            ctx->adj_ws = nullptr;
            cudaGetLastError();
            return afail(ctx, RTPN_ENOMEM, "adjoint: device memory for checkpoints and segment states");
        }
        ctx->adj_ws_bytes = total;
    }
    char* ws = (char*)ctx->adj_ws;
    char *ck = ws + off[CK], *ring = ws + off[RING], *lam = ws + off[LAM], *wbuf = ws + off[WB];
    char *dfac = ws + off[DFAC], *gacc = ws + off[GACC], *gqb = ws + off[GQ], *part = ws + off[PART];
    char *maps = ws + off[MAPS], *tabs = ws + off[TABS];
    auto X = [&](int sg, int i) -> char* {
        return i == 0 ? ck + (size_t)sg * state : ring + (size_t)(i - 1) * state;
    };
    auto XM = [&](int sg, int i) -> const char* { return maps + (size_t)(i == 0 ? sg : nseg + i - 1) * mapb; };
    // tensor maps over every checkpoint and ring state, unless the last call built the same ones
    const long long key[4] = {nseg, nring, ctx->stage_variant, (long long)(size_t)ws};
    if (!std::equal(key, key + 4, ctx->adj_maps_key)) {
        std::fill(ctx->adj_maps_key, ctx->adj_maps_key + 4, -1);
        for (int sg = 0; sg < nseg; ++sg)
            if (stage_maps_for(ctx, X(sg, 0), maps + (size_t)sg * mapb))
                return afail(ctx, RTPN_ECUDA, "adjoint: tensor maps");
        for (int i = 1; i <= nring; ++i)
            if (stage_maps_for(ctx, X(0, i), maps + (size_t)(nseg + i - 1) * mapb))
                return afail(ctx, RTPN_ECUDA, "adjoint: tensor maps");
        std::copy(key, key + 4, ctx->adj_maps_key);
    }
    if (cudaMemcpyAsync(tabs, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return afail(ctx, RTPN_ECUDA, "adjoint: tables");
    k_adj_factors<float><<<blocks_for(V), 256, 0, st>>>(ctx->media, ctx->media + V, (float*)dfac, g, ctx->dt);

    auto seg_steps = [&](int sg) { return std::min(k, (sg + 1) * ckpt) - sg * ckpt; };
    auto pass_cls = [](int j) { return (j & 1) ? 0 : 1; };
    auto pass_ofs = [](int j, int m) { return (j == 0 || j == 2 * m) ? FAC_HALF : FAC_FULL; };
    auto run_segment = [&](int sg) -> int {
        const int m = seg_steps(sg);
        for (int j = 0; j <= 2 * m; ++j) {
            const int rc = launch_stage_between(ctx, pass_cls(j), pass_ofs(j, m), XM(sg, (j + 1) / 2), XM(sg, j / 2),
                                                X(sg, j / 2 + 1), st);
            if (rc) return afail(ctx, RTPN_ECUDA, std::string("adjoint: staged pass: ") +
                                                      cudaGetErrorString((cudaError_t)rc));
        }
        return RTPN_OK;
    };

    // ---- forward: segment by segment; each end state (even class in X[m], odd class in X[m + 1])
    // is the next checkpoint, the last one the context's state
    const size_t even_b = (size_t)ne * V * sizeof(float), odd_b = (size_t)no * V * sizeof(float);
    if (nseg > 0) cudaMemcpyAsync(X(0, 0), ctx->u, state, cudaMemcpyDeviceToDevice, st);
    for (int sg = 0; sg < nseg; ++sg) {
        if (int rc = run_segment(sg)) return rc;
        const int m = seg_steps(sg);
        char* dst = sg + 1 < nseg ? X(sg + 1, 0) : (char*)ctx->u;
        cudaMemcpyAsync(dst, X(sg, m), even_b, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(dst + even_b, X(sg, m + 1) + even_b, odd_b, cudaMemcpyDeviceToDevice, st);
    }
    ctx->steps_done += k;  // the context now holds u(k), whatever the backward sweep meets
    // J = sum w u_0 (u_0 is internal component 0)
    k_dot_u0<float><<<1024, 256, 0, st>>>((const float*)ctx->u, w_dev, V, (double*)part);
    launch_sum<double>((const double*)part, 1024, ctx->partial, 1, ctx->partial + SUM_BLOCKS, st);
    cudaMemcpyAsync(J, ctx->partial + SUM_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, st);

    // ---- backward, pass by pass in reverse
    float* lp = (float*)lam;
    cudaMemsetAsync(lp, 0, state, st);
    k_copy_cast<double, float><<<1024, 256, 0, st>>>(w_dev, lp, V);  // lam_0 = w
    cudaMemsetAsync(gacc, 0, (size_t)9 * V * sizeof(double), st);
    cudaMemsetAsync(gqb, 0, (size_t)V * sizeof(double), st);
    const int* tp = (const int*)tabs;
    // pend[c]: the factor offset of the last pulled-back pass on class c whose lam_c <- alpha lam_c
    // is still to come (folded into the next transposed coupling onto class c), -1 for none
    int pend[2] = {-1, -1};
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int m = seg_steps(sg);
        if (sg < nseg - 1)
            if (int rc = run_segment(sg)) return rc;
        for (int j = 2 * m; j >= 0; --j) {
            const int cls = pass_cls(j), ofs = pass_ofs(j, m);
            const size_t a0 = cls == 0 ? 0 : (size_t)ne * V;
            const int ng = (int)pt[cls].grp.size() / 4;
            const float* pre = (const float*)X(sg, j / 2) + a0;
            const float* post = (const float*)X(sg, j / 2 + 1) + a0;
            k_adj_pull<<<blocks_for(V / 4), 256, 0, st>>>(pre, post, lp + a0, (float*)wbuf, (const float*)ctx->fac,
                                                          (const float*)dfac, ofs, pend[cls], tp + at[cls][0], ng,
                                                          tp + at[cls][1], V, (double*)gacc, (double*)gqb);
            pend[cls] = ofs;
            const int rc = launch_stage_adjoint_sources(ctx, 1 - cls, lp, (const float*)wbuf, std::max(ne, no),
                                                        pend[1 - cls], st);
            if (rc) return afail(ctx, RTPN_ECUDA, "adjoint: staged transposed coupling failed");
            pend[1 - cls] = -1;
        }
    }
    k_adj_media<<<blocks_for(V), 256, 0, st>>>((const double*)gacc, g, gsa, gss);
    cudaMemcpyAsync(gq_out, gqb, (size_t)V * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return afail(ctx, RTPN_ECUDA, std::string("adjoint: ") + cudaGetErrorString(e));
    if (int rc = rtpn_synchronize(ctx)) return rc;  // also reports a staged wait that ran out
    return RTPN_OK;
}

}  // namespace

extern "C" int rtpn_adjoint(rtpn_ctx* ctx, const void* w, int dtype, int where, int k, int ckpt_every,
                            double* g_sa, double* g_ss, double* g_q, int out_where, double* J) {
    if (!ctx || !w || !g_sa || !g_ss || !g_q || !J || k < 0 || ckpt_every < 1) return RTPN_EINVAL;
    if ((dtype != RTPN_DTYPE_F64 && dtype != RTPN_DTYPE_F32) || (where != RTPN_HOST && where != RTPN_DEVICE) ||
        (out_where != RTPN_HOST && out_where != RTPN_DEVICE))
        return afail(ctx, RTPN_EINVAL, "adjoint: bad dtype/where");
    if (ctx->prec == RTPN_BF16) return afail(ctx, RTPN_EUNSUPPORTED, "adjoint: BF16 storage");
    if (ctx->scat) return afail(ctx, RTPN_EUNSUPPORTED, "adjoint: anisotropic scattering");
    if (!ctx->media_set || !ctx->media) return afail(ctx, RTPN_ESTATE, "adjoint: media not set");
    const long long V = ctx->g.V;
    // the weights and outputs as FP64 device arrays
    Buf wd, out;
    if (!wd.alloc((size_t)V * sizeof(double)) || !out.alloc((size_t)3 * V * sizeof(double)))
        return afail(ctx, RTPN_ENOMEM, "adjoint: buffers");
    if (dtype == RTPN_DTYPE_F64) {
        cudaMemcpyAsync(wd.p, w, V * sizeof(double),
                        where == RTPN_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream);
    } else {
        Buf tmp;
        if (!tmp.alloc((size_t)V * sizeof(float))) return afail(ctx, RTPN_ENOMEM, "adjoint: buffers");
        cudaMemcpyAsync(tmp.p, w, V * sizeof(float),
                        where == RTPN_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream);
        launch_convert<float, double>((const float*)tmp.p, (double*)wd.p, V, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
    }
    double* o = (double*)out.p;
    int rc = ctx->prec == RTPN_FP64
                 ? adjoint_impl<double, double>(ctx, (const double*)wd.p, k, ckpt_every, o, o + V, o + 2 * V, J)
                 : ctx->active_kernel == RTPN_KERNEL_STAGE
                     ? adjoint_staged(ctx, (const double*)wd.p, k, ckpt_every, o, o + V, o + 2 * V, J)
                     : adjoint_impl<float, float>(ctx, (const double*)wd.p, k, ckpt_every, o, o + V, o + 2 * V, J);
    if (rc) return rc;
    const cudaMemcpyKind kind = out_where == RTPN_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    double* dst[3] = {g_sa, g_ss, g_q};
    for (int i = 0; i < 3; ++i) cudaMemcpyAsync(dst[i], o + (size_t)i * V, V * sizeof(double), kind, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return afail(ctx, RTPN_ECUDA, cudaGetErrorString(e));
    return RTPN_OK;
}

extern "C" int rtpn_adjoint_release(rtpn_ctx* ctx) {
    if (!ctx) return RTPN_EINVAL;
    if (ctx->adj_ws) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e == cudaSuccess) e = cudaFree(ctx->adj_ws);
        ctx->adj_ws = nullptr;
        ctx->adj_ws_bytes = 0;
        std::fill(ctx->adj_maps_key, ctx->adj_maps_key + 4, -1);
        if (e != cudaSuccess) return afail(ctx, RTPN_ECUDA, std::string("adjoint release: ") + cudaGetErrorString(e));
    }
    return RTPN_OK;
}

extern "C" int rtpn_detector(rtpn_ctx* ctx, const void* w, int dtype, int where, double* J, int J_where) {
    if (!ctx || !w || !J) return RTPN_EINVAL;
    if ((dtype != RTPN_DTYPE_F64 && dtype != RTPN_DTYPE_F32) || (where != RTPN_HOST && where != RTPN_DEVICE) ||
        (J_where != RTPN_HOST && J_where != RTPN_DEVICE))
        return afail(ctx, RTPN_EINVAL, "detector: bad dtype/where");
    const long long V = ctx->g.V;
    cudaStream_t st = ctx->stream;
    // the weights as FP64 on the device: used in place, or widened into the context's FP64 staging plane
    const double* wd = (const double*)w;
    Buf tmp;
    if (dtype == RTPN_DTYPE_F64 && where == RTPN_HOST) {
        cudaMemcpyAsync(ctx->staging, w, (size_t)V * 8, cudaMemcpyHostToDevice, st);
        wd = (const double*)ctx->staging;
    } else if (dtype == RTPN_DTYPE_F32) {
        const float* wf = (const float*)w;
        if (where == RTPN_HOST) {
            if (!tmp.alloc((size_t)V * 4)) return afail(ctx, RTPN_ENOMEM, "detector: weights");
            cudaMemcpyAsync(tmp.p, w, (size_t)V * 4, cudaMemcpyHostToDevice, st);
            wf = (const float*)tmp.p;
        }
        launch_convert<float, double>(wf, (double*)ctx->staging, V, st);
        wd = (const double*)ctx->staging;
    }
    if (ctx->prec == RTPN_FP64)
        k_dot_u0<double><<<SUM_BLOCKS, 256, 0, st>>>((const double*)ctx->u, wd, V, ctx->partial);
    else if (ctx->prec == RTPN_FP32)
        k_dot_u0<float><<<SUM_BLOCKS, 256, 0, st>>>((const float*)ctx->u, wd, V, ctx->partial);
    else
        k_dot_u0<__nv_bfloat16><<<SUM_BLOCKS, 256, 0, st>>>((const __nv_bfloat16*)ctx->u, wd, V, ctx->partial);
    k_partials_total<<<1, 1024, 0, st>>>(ctx->partial, SUM_BLOCKS, ctx->partial + SUM_BLOCKS);
    cudaError_t e = cudaMemcpyAsync(J, ctx->partial + SUM_BLOCKS, sizeof(double),
                                    J_where == RTPN_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && (J_where == RTPN_HOST || tmp.p)) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return afail(ctx, RTPN_ECUDA, std::string("detector: ") + cudaGetErrorString(e));
    return RTPN_OK;
}
