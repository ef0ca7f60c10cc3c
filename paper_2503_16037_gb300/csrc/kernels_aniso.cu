// Anisotropic multiple scattering (the edge unknowns of Eq. flux_system; see
// aniso.h for the recurrence and its factored form).  Layouts: X and Xn are
// [nin][n_nodes] (plane per arrival direction, rows = node ids), the
// per-node tables are transposed ([direction][node]) so that a warp's 32
// nodes read and write 128 contiguous bytes, L is haloed [nd][npad] so the
// transport pass reads it at the source-relative positions of the slot
// descriptors, and val holds the raw deposit fractions P in K's slot-major
// layout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "aniso.h"
#include "aniso_contract.cuh"
#include "asm_util.cuh"
#include "kern.h"
#include "stage.cuh"

namespace tk {

// HG of species sp summed over the lattice points of the cell of direction u,
// the angle measured from arrival direction w: one warp per (u, w, sp)
__global__ void k_aniso_qcells(GridC g, ViewC vc, ViewP vp, double *Qraw) {
    const int nin = g.nd + g.ngd;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long long)g.S * nin * g.nd) return;  // whole warps
    const int u = (int)(wid % g.nd), w = (int)((wid / g.nd) % nin), sp = (int)(wid / ((long long)g.nd * nin));
    const double *wh = vp.dirhat + 3 * w;
    double acc = 0.0;
    for (int m = vp.cell_start[u] + lane; m < vp.cell_start[u + 1]; m += 32) {
        const double *s = vp.lattice + 3 * (size_t)m;
        acc += hg<double>(vc.g[sp], wh[0] * s[0] + wh[1] * s[1] + wh[2] * s[2]);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) Qraw[((size_t)sp * nin + w) * g.nd + u] = acc;
}

// each row (sp, w) divided by its sum over the cells
template <typename T>
__global__ void k_aniso_qnorm(GridC g, const double *Qraw, T *Q) {
    const int nin = g.nd + g.ngd;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.S * nin) return;
    const double *row = Qraw + (size_t)r * g.nd;
    double t = 0.0;
    for (int u = 0; u < g.nd; ++u) t += row[u];
    for (int u = 0; u < g.nd; ++u) Q[(size_t)r * g.nd + u] = (T)(row[u] / t);
}


// SQ[z][sp][w]: Q_sp(w -> u) summed over the directions u that have a
// receiver from layer z (all but the upward ones that leave the top)
template <typename T>
__global__ void k_ani_sq(GridC g, GraphP gp, const T *Q, T *SQ) {
    const int nin = g.nd + g.ngd;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.nz * g.S * nin) return;
    const int w = idx % nin, sp = (idx / nin) % g.S, z = idx / (nin * g.S);
    const T *row = Q + ((size_t)sp * nin + w) * g.nd;
    T s = T(0);
    for (int u = 0; u < g.nd; ++u)
        if (z + gp.dirs[u].z < g.nz) s += row[u];
    SQ[idx] = s;
}

// Couplings of every chain (transposed, 0 where the chain has no receiver),
// whether the routing applies at each node, the first-order leaving power
// and the ground sources' weights (one thread per node; the couplings as in
// the node form's normalisers, the sun weights and routing as the assembly
// applies them).
template <typename T>
__global__ void k_aniso_couple(GridC g, GraphP gp, FieldP<T> f, ViewC vc, AniP<T> a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_nodes) return;
    const T rt_lamb = dsqrt<T>((T)(vc.albedo * __longlong_as_double((long long)*f.mus_max_bits)));
    const int z = j / g.nxy, r = j - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    T *Ls = a.LsT + j;  // plane stride n_nodes
    if (j < g.n_atm) {
        const T rt_src = f.rt[j];
        T w[MAX_SPECIES];
        for (int sp = 0; sp < g.S; ++sp) w[sp] = f.wsp[(size_t)sp * g.n_atm + j];
        T sq = 0, sqc = 0;
        bool any = false;
        for (int u = 0; u < g.nd; ++u) {
            const int4 d = gp.dirs[u];
            const int rz = z + d.z;
            T C = T(-1);
            if (rz < g.nz) {
                T rtn, dist;
                if (rz >= 0) {
                    rtn = f.rt[(rz * g.ny + wrap_small(y + d.y, g.ny)) * g.nx + wrap_small(x + d.x, g.nx)];
                    dist = Cst<T>::dir_len(gp, u);
                } else {
                    rtn = rt_lamb;
                    dist = ((T)z + T(0.5)) / (T)(-d.z) * Cst<T>::dir_len(gp, u);
                }
                C = rt_src * rtn / dist;
            }
            a.CT[(size_t)u * g.n_atm + j] = C > T(0) ? C : T(0);
            any = any || C > T(0);
            T qs = 0;
            for (int sp = 0; sp < g.S; ++sp) qs += w[sp] * f.q_sun[sp * g.nd + u];
            if (C >= T(0)) {
                sq += qs;
                sqc += qs * C;
            }
        }
        a.on[j] = (vc.coupling && any) ? T(1) : T(0);
        const bool on = vc.coupling && sqc > T(0);
        const T e1 = f.e1[j];
        for (int u = 0; u < g.nd; ++u) {
            T qs = 0;
            for (int sp = 0; sp < g.S; ++sp) qs += w[sp] * f.q_sun[sp * g.nd + u];
            const T C = a.CT[(size_t)u * g.n_atm + j];
            const bool has = z + gp.dirs[u].z < g.nz;
            Ls[(size_t)u * g.n_nodes] = e1 * qs * ((on && has) ? C * sq / sqc : T(1));
        }
    } else {
        const int c = j - g.n_atm;
        T sq = 0, sqc = 0;
        T Cv[128];
        for (int k = 0; k < g.ngd; ++k) {
            const int4 m = gp.gmem1[k];
            T C = T(-1);
            if (m.z <= g.nz) {
                const T rtn = f.rt[((m.z - 1) * g.ny + wrap_small(y + m.y, g.ny)) * g.nx + wrap_small(x + m.x, g.nx)];
                C = rt_lamb * rtn / Cst<T>::gdist1(gp, k);
            }
            Cv[k] = C;
            const T q = Cst<T>::q_lamb(gp, k);
            if (C >= T(0)) {
                sq += q;
                sqc += q * C;
            }
        }
        const bool on = vc.coupling && sqc > T(0);
        const T e1 = f.e1[j];
        for (int k = 0; k < g.ngd; ++k) {
            const T C = Cv[k];
            const T wg = Cst<T>::q_lamb(gp, k) * ((on && C >= T(0)) ? C * sq / sqc : T(1));
            a.Wg[(size_t)c * g.ngd + k] = wg;
            Ls[(size_t)k * g.n_nodes] = e1 * wg;
        }
    }
}

// Leaving power of the ground (Lambertian) nodes: the total X times the
// ground weights, plus Lsun where `sun` is set
template <typename T, typename XT, typename LT>
__global__ void k_ani_ground(GridC g, AniP<T> a, const XT *__restrict__ X, LT *Lh, int sun, const int *ctl) {
    if (ctl && *(volatile const int *)ctl) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.n_ground) return;
    const int j = g.n_atm + c, y = c / g.nx, x = c - y * g.nx;
    const int nin = g.nd + g.ngd;
    XT xt = XT(0);
    for (int w = 0; w < nin; ++w) xt += X[(size_t)w * g.n_nodes + j];
    for (int k = 0; k < g.ngd; ++k) {
        LT l = (LT)xt * (LT)a.Wg[(size_t)c * g.ngd + k];
        if (sun) l += (LT)a.LsT[(size_t)k * g.n_nodes + j];
        store_halo(Lh + (size_t)k * g.npad, g, x, y, g.nz, l);
    }
}

// Transport as a gather: block = one group of 128 receiver rows (the edge
// kernel's lane quads), warp w sums the arrival directions w, w + kAniW, ...
// over the template's slots of that direction (tperm / tseg order), so
// every X(i, w) is written once, in a fixed order.
//   MODE 0: Xn = [radd] + rho sum P L, and the change against Xold
//   MODE 1: Xn = rho sum P L64 - X64 (FP64 sums, the residual stored in FP32)
// Per-block sums of the squared change (residual) and of the squares of Xn
// (X64) go to a.part.
constexpr int kAniW = 4;
template <typename T, int MODE, typename LT, typename XT>
__global__ void __launch_bounds__(32 * kAniW) k_ani_transport(GridC g, GraphP gp, FieldP<T> f, ViewC vc, AniP<T> a,
                                                              const LT *__restrict__ Lh,
                                                              const XT *__restrict__ Xold, T *Xn,
                                                              const T *__restrict__ radd) {
    __shared__ double red[2][kAniW];
    if (MODE == 0 && *(volatile const int *)a.ctl) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nin = g.nd + g.ngd;
    const GroupRows G = group_rows(g, gp, blockIdx.x);
    const bool ground_row = G.z == g.nz;
    T rho[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (G.row[k] < 0) {
            rho[k] = T(0);
        } else if (!ground_row) {
            const T me = f.mu_e[G.row[k]], ms = f.mu_st[G.row[k]];
            rho[k] = me > T(0) ? ms / me : T(0);
        } else {
            rho[k] = (T)vc.albedo;
        }
    }
    const T *vrow = f.val + G.vb + 4 * lane;
    const int *perm = a.tperm + G.t0;
    const int *seg = a.tseg + (size_t)G.z * (nin + 1);
    double d2 = 0.0, n2 = 0.0;
    for (int d = w; d < nin; d += kAniW) {
        const int e0 = __ldg(seg + d), e1 = __ldg(seg + d + 1);
        LT acc[4] = {LT(0), LT(0), LT(0), LT(0)};
        for (int e = e0; e < e1; ++e) {
            const int t = __ldg(perm + e);
            const ASlot &sd = gp.aslot[G.t0 + t];
            const int src = __ldg(&sd.src), dir = __ldg(&sd.dir);
            T P[4];
            ld_quad(vrow + (size_t)t * kGroup, P);
            const LT *Ld = Lh + (size_t)dir * g.npad + src;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (G.row[k] >= 0) acc[k] += (LT)P[k] * __ldg(Ld + G.rp[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (G.row[k] < 0) continue;
            const size_t q = (size_t)d * g.n_nodes + G.row[k];
            if constexpr (MODE == 0) {
                T xn = rho[k] * (T)acc[k];
                if (radd) xn += radd[q];
                const double dx = (double)xn - (double)Xold[q];
                Xn[q] = xn;
                d2 += dx * dx;
                n2 += (double)xn * (double)xn;
            } else {
                const double xo = (double)Xold[q];
                const double r = (double)rho[k] * (double)acc[k] - xo;
                Xn[q] = (T)r;
                d2 += r * r;
                n2 += xo * xo;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if (lane == 0) {
        red[0][w] = d2;
        red[1][w] = n2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < kAniW; ++i) {
            s0 += red[0][i];
            s1 += red[1][i];
        }
        a.part[2 * (size_t)blockIdx.x] = s0;
        a.part[2 * (size_t)blockIdx.x + 1] = s1;
    }
}

// Sums of the blocks' partials in a fixed order; a series term sets the
// converged flag when its relative change is at most tol (and does nothing
// once the flag is set).
__global__ void k_ani_check(const double *part, int nblk, double *acc, int *ctl, double tol, int term, int series) {
    __shared__ double s0[256], s1[256];
    if (series && *(volatile int *)ctl) return;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblk; i += 256) {
        a += part[2 * (size_t)i];
        b += part[2 * (size_t)i + 1];
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            s0[threadIdx.x] += s0[threadIdx.x + h];
            s1[threadIdx.x] += s1[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double rel = s1[0] > 0.0 ? sqrt(s0[0] / s1[0]) : 0.0;
        acc[0] = s0[0];
        acc[1] = s1[0];
        acc[2] = rel;
        if (series && rel <= tol) {
            ctl[0] = 1;
            ctl[1] = term;
        }
    }
}

__global__ void k_ani_update(long long n, const float *e, double *X64, int init) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        X64[i] = init ? (double)e[i] : X64[i] + (double)e[i];
}

// x = sum_w X(i, w) into the FP64 haloed vector, and the emission toward the
// instrument E_i = e1_i Theta_i(s0 . v) + sum_w Theta_i(w . v) X(i, w)
template <typename T, typename XT>
__global__ void k_aniso_finish(GridC g, FieldP<T> f, const XT *__restrict__ X, double *x64, T *emis) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_nodes) return;
    const int nin = g.nd + g.ngd;
    const int z = i / g.nxy, r = i - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    double xt = 0.0;
    for (int wv = 0; wv < nin; ++wv) xt += (double)X[(size_t)wv * g.n_nodes + i];
    store_halo(x64, g, x, y, z, xt);
    if (i >= g.n_atm) return;
    double w[MAX_SPECIES];
    double th0 = 0;
    for (int sp = 0; sp < g.S; ++sp) {
        w[sp] = (double)f.wsp[(size_t)sp * g.n_atm + i];
        th0 += w[sp] * (double)f.hg0v[sp];
    }
    double e = 0;
    for (int wv = 0; wv < nin; ++wv) {
        const double xw = (double)X[(size_t)wv * g.n_nodes + i];
        if (xw == 0.0) continue;
        double th = 0;
        for (int sp = 0; sp < g.S; ++sp) th += w[sp] * (double)f.hgv[sp * nin + wv];
        e += th * xw;
    }
    emis[i] = (T)((double)f.e1[i] * th0 + e);
}

// ---- launchers ----
namespace {

// tensor-core launch of the leave contraction: N padded to one of a few
// tile widths (N <= 128), S <= MAX_SPECIES
template <class Op>
void mma_leave(cudaStream_t st, const Op &op, int S, int R, int N, const float *B, const int *ctl, int *status) {
    const int np = ani_leave_np(N, S);
#define TK_L(SS, NN) ani_mma_launch<SS, NN, Op>(st, op, R, N, B, ctl, status)
    if (S == 1) {
        if (np == 32) TK_L(1, 32); else if (np == 64) TK_L(1, 64); else if (np == 112) TK_L(1, 112); else TK_L(1, 128);
    } else if (S == 2) {
        if (np == 32) TK_L(2, 32); else if (np == 64) TK_L(2, 64); else if (np == 112) TK_L(2, 112); else TK_L(2, 128);
    } else if (S == 3) {
        TK_L(3, 128);
    } else {
        TK_L(4, 128);
    }
#undef TK_L
}

// first node of the layers from which some direction has no receiver
// (the top max(uz) layers)
inline int top_begin(const GridC &g) { return std::max(0, g.nz - g.R) * g.nxy; }

template <typename T>
LeaveOp<T, T, T> leave_op(const GridC &g, const GraphP &gp, const AniP<T> &a, const T *wsp, const T *X, int sun,
                          int top) {
    LeaveOp<T, T, T> op;
    op.g = g;
    op.jbeg = top ? top_begin(g) : 0;
    op.top = top;
    op.dirs = gp.dirs;
    op.zf = a.zf;
    op.wsp = wsp;
    op.CT = a.CT;
    op.on = a.on;
    op.LsT = a.LsT;
    op.Q = a.Q;
    op.X = X;
    op.Lh = a.Lh;
    op.sun = sun;
    return op;
}
template <typename T>
SqcOp<T> sqc_op(const GridC &g, const AniP<T> &a, const T *wsp) {
    SqcOp<T> op;
    op.g = g;
    op.jbeg = 0;
    op.CT = a.CT;
    op.wsp = wsp;
    op.on = a.on;
    op.SQ = a.SQ;
    op.Q = a.Q;
    op.zf = a.zf;
    return op;
}

// the contractions with their raw outputs out[n][n_atm] (tests)
template <class Base>
struct RawOp : Base {
    float *raw;
    struct Pre {};
    __device__ __forceinline__ Pre pre(int) const { return Pre{}; }
    template <typename V>
    __device__ __forceinline__ void out(const Pre &, int j, int n, V val) const {
        raw[(size_t)n * this->g.n_atm + j] = (float)val;
    }
};

}  // namespace

template <typename T>
void launch_aniso_prep(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const ViewP &vp, const AniP<T> &a, long long *launches) {
    const int nin = g.nd + g.ngd;
    const long long warps = (long long)g.S * nin * g.nd;
    k_aniso_qcells<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(g, vc, vp, a.Qraw);
    k_aniso_qnorm<T><<<(g.S * nin + 127) / 128, 128, 0, st>>>(g, a.Qraw, a.Q);
    k_ani_sq<T><<<(g.nz * g.S * nin + 127) / 128, 128, 0, st>>>(g, gp, a.Q, a.SQ);
    k_aniso_couple<T><<<(g.n_nodes + 127) / 128, 128, 0, st>>>(g, gp, f, vc, a);
    // the routing denominators on the CUDA cores: zf is part of the operator
    // the FP64 residual refines against, so it keeps FP32 sums
    ani_simt_launch<T, 0>(st, sqc_op<T>(g, a, f.wsp), g.S, g.nd, nin, nullptr);
    if (launches) *launches += 5;
    if constexpr (sizeof(T) == 4) {
        if (a.mma) {
            const LeaveOp<T, T, T> lop = leave_op<T>(g, gp, a, f.wsp, nullptr, 1, 0);
            k_ani_pack<<<256, 256, 0, st>>>(lop, g.S, nin, g.nd, ani_leave_np(g.nd, g.S), a.Bl);
            if (launches) *launches += 1;
        }
    }
}

template <typename T>
void launch_aniso_term(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const AniP<T> &a, const T *X, T *Xn, const T *radd, bool sun, double tol, int term,
                       long long *launches) {
    const int nin = g.nd + g.ngd;
    const LeaveOp<T, T, T> lop = leave_op<T>(g, gp, a, f.wsp, X, sun ? 1 : 0, 0);
    const LeaveOp<T, T, T> top = leave_op<T>(g, gp, a, f.wsp, X, sun ? 1 : 0, 1);
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        if (a.mma) {
            mma_leave(st, lop, g.S, nin, g.nd, a.Bl, a.ctl, f.status);
            mma_leave(st, top, g.S, nin, g.nd, a.Bl, a.ctl, f.status);
            done = true;
        }
    }
    if (!done) {
        ani_simt_launch<T, 0>(st, lop, g.S, nin, g.nd, a.ctl);
        ani_simt_launch<T, 0>(st, top, g.S, nin, g.nd, a.ctl);
    }
    if (g.n_ground > 0)
        k_ani_ground<T, T, T><<<(g.n_ground + 127) / 128, 128, 0, st>>>(g, a, X, a.Lh, sun ? 1 : 0, a.ctl);
    const int nblk = (g.nz + 1) * g.gpl;
    k_ani_transport<T, 0, T, T><<<nblk, 32 * kAniW, 0, st>>>(g, gp, f, vc, a, a.Lh, X, Xn, radd);
    k_ani_check<<<1, 256, 0, st>>>(a.part, nblk, a.acc, a.ctl, tol, term, 1);
    if (launches) *launches += g.n_ground > 0 ? 5 : 4;
}

void launch_aniso_resid(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<float> &f,
                        const ViewC &vc, const AniP<float> &a, const double *X64, double *L64, float *r,
                        long long *launches) {
    const int nin = g.nd + g.ngd;
    LeaveOp<float, double, double> op;
    op.g = g;
    op.jbeg = 0;
    op.top = 0;
    op.dirs = gp.dirs;
    op.zf = a.zf;
    op.wsp = f.wsp;
    op.CT = a.CT;
    op.on = a.on;
    op.LsT = a.LsT;
    op.Q = a.Q;
    op.X = X64;
    op.Lh = L64;
    op.sun = 1;
    ani_simt_launch<float, 1>(st, op, g.S, nin, g.nd, nullptr);
    op.top = 1;
    op.jbeg = top_begin(g);
    ani_simt_launch<float, 1>(st, op, g.S, nin, g.nd, nullptr);
    if (g.n_ground > 0)
        k_ani_ground<float, double, double><<<(g.n_ground + 127) / 128, 128, 0, st>>>(g, a, X64, L64, 1, nullptr);
    const int nblk = (g.nz + 1) * g.gpl;
    k_ani_transport<float, 1, double, double><<<nblk, 32 * kAniW, 0, st>>>(g, gp, f, vc, a, L64, X64, r, nullptr);
    k_ani_check<<<1, 256, 0, st>>>(a.part, nblk, a.acc, a.ctl, 0.0, 0, 0);
    if (launches) *launches += g.n_ground > 0 ? 5 : 4;
}

void launch_aniso_update(cudaStream_t st, long long n, const float *e, double *X64, bool init) {
    k_ani_update<<<1216, 256, 0, st>>>(n, e, X64, init ? 1 : 0);
}

template <typename T, typename XT>
void launch_aniso_finish(cudaStream_t st, const GridC &g, const FieldP<T> &f, const XT *X, double *x64, T *emis,
                         long long *launches) {
    k_aniso_finish<T, XT><<<(g.n_nodes + 127) / 128, 128, 0, st>>>(g, f, X, x64, emis);
    if (launches) *launches += 1;
}

void launch_aniso_contract_test(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<float> &f,
                                const AniP<float> &a, const float *X, float *out, int which, bool mma) {
    const int nin = g.nd + g.ngd;
    if (which == 0) {
        RawOp<LeaveOp<float, float, float>> op;
        static_cast<LeaveOp<float, float, float> &>(op) = leave_op<float>(g, gp, a, f.wsp, X, 0, 0);
        op.raw = out;
        if (mma) mma_leave(st, op, g.S, nin, g.nd, a.Bl, nullptr, f.status);
        else ani_simt_launch<float, 0>(st, op, g.S, nin, g.nd, nullptr);
    } else {
        RawOp<SqcOp<float>> op;
        static_cast<SqcOp<float> &>(op) = sqc_op<float>(g, a, f.wsp);
        op.raw = out;
        ani_simt_launch<float, 0>(st, op, g.S, g.nd, nin, nullptr);
    }
}

#define INST(T)                                                                                                 \
    template void launch_aniso_prep<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,          \
                                       const ViewC &, const ViewP &, const AniP<T> &, long long *);             \
    template void launch_aniso_term<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,          \
                                       const ViewC &, const AniP<T> &, const T *, T *, const T *, bool, double, \
                                       int, long long *);                                                       \
    template void launch_aniso_finish<T, T>(cudaStream_t, const GridC &, const FieldP<T> &, const T *,          \
                                            double *, T *, long long *);
INST(float)
INST(double)
#undef INST
template void launch_aniso_finish<float, double>(cudaStream_t, const GridC &, const FieldP<float> &,
                                                 const double *, double *, float *, long long *);

}  // namespace tk
