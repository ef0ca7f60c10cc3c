// Anisotropic multiple scattering (the edge unknowns of Eq. flux_system; see
// aniso.h for the recurrence).  Layouts: X and Xn are [nin][n_nodes] (plane
// per arrival direction, rows = node ids), L is haloed [nd][npad] so the
// transport pass reads it at the source-relative positions of the slot
// descriptors, and val holds the raw deposit fractions P in K's slot-major
// layout.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "aniso.h"
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

// Couplings of every chain, the first-order leaving power and the ground
// sources' weights (one thread per node; the couplings as in the node form's
// normalisers, the sun weights and routing as the assembly applies them).
template <typename T>
__global__ void k_aniso_couple(GridC g, GraphP gp, FieldP<T> f, ViewC vc, AniP<T> a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_nodes) return;
    const T rt_lamb = dsqrt<T>((T)(vc.albedo * __longlong_as_double((long long)*f.mus_max_bits)));
    const int z = j / g.nxy, r = j - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    T *Cj = a.C + (size_t)j * g.nd;
    T *Ls = a.Lsun + (size_t)j * g.nd;
    if (j < g.n_atm) {
        const T rt_src = f.rt[j];
        T w[MAX_SPECIES];
        for (int sp = 0; sp < g.S; ++sp) w[sp] = f.wsp[(size_t)sp * g.n_atm + j];
        T sq = 0, sqc = 0;
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
            Cj[u] = C;
            T qs = 0;
            for (int sp = 0; sp < g.S; ++sp) qs += w[sp] * f.q_sun[sp * g.nd + u];
            if (C >= T(0)) {
                sq += qs;
                sqc += qs * C;
            }
        }
        const bool on = vc.coupling && sqc > T(0);
        const T e1 = f.e1[j];
        for (int u = 0; u < g.nd; ++u) {
            T qs = 0;
            for (int sp = 0; sp < g.S; ++sp) qs += w[sp] * f.q_sun[sp * g.nd + u];
            const T C = Cj[u];
            Ls[u] = e1 * qs * ((on && C >= T(0)) ? C * sq / sqc : T(1));
        }
    } else {
        const int c = j - g.n_atm;
        T sq = 0, sqc = 0;
        for (int k = 0; k < g.ngd; ++k) {
            const int4 m = gp.gmem1[k];
            T C = T(-1);
            if (m.z <= g.nz) {
                const T rtn = f.rt[((m.z - 1) * g.ny + wrap_small(y + m.y, g.ny)) * g.nx + wrap_small(x + m.x, g.nx)];
                C = rt_lamb * rtn / Cst<T>::gdist1(gp, k);
            }
            Cj[k] = C;
            const T q = Cst<T>::q_lamb(gp, k);
            if (C >= T(0)) {
                sq += q;
                sqc += q * C;
            }
        }
        const bool on = vc.coupling && sqc > T(0);
        const T e1 = f.e1[j];
        for (int k = 0; k < g.ngd; ++k) {
            const T C = Cj[k];
            const T wg = Cst<T>::q_lamb(gp, k) * ((on && C >= T(0)) ? C * sq / sqc : T(1));
            a.Wg[(size_t)c * g.ngd + k] = wg;
            Ls[k] = e1 * wg;
        }
    }
}

// Leaving power of every source along each of its directions: one warp per
// node, lane l handles directions l + 32 k.
constexpr int kAniU = 4;  // directions per lane (nd <= 128)
template <typename T>
__global__ void k_aniso_leave(GridC g, GraphP gp, FieldP<T> f, ViewC vc, AniP<T> a, const T *__restrict__ X) {
    const int nin = g.nd + g.ngd;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= g.n_nodes) return;  // whole warps
    const int z = j / g.nxy, r = j - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    const T *Cj = a.C + (size_t)j * g.nd;
    const T *Ls = a.Lsun + (size_t)j * g.nd;
    T acc[kAniU];
    if (j < g.n_atm) {
        T w[MAX_SPECIES];
        for (int sp = 0; sp < g.S; ++sp) w[sp] = f.wsp[(size_t)sp * g.n_atm + j];
        T C[kAniU];
#pragma unroll
        for (int k = 0; k < kAniU; ++k) {
            const int u = lane + 32 * k;
            acc[k] = u < g.nd ? Ls[u] : T(0);
            C[k] = u < g.nd ? Cj[u] : T(-1);
        }
        for (int wv = 0; wv < nin; ++wv) {
            const T xw = X[(size_t)wv * g.n_nodes + j];
            if (xw == T(0)) continue;  // the same for the whole warp
            T q[kAniU];
            T sq = 0, sqc = 0;
#pragma unroll
            for (int k = 0; k < kAniU; ++k) {
                const int u = lane + 32 * k;
                T v = 0;
                if (u < g.nd)
                    for (int sp = 0; sp < g.S; ++sp) v += w[sp] * a.Q[((size_t)sp * nin + wv) * g.nd + u];
                q[k] = v;
                if (C[k] >= T(0)) {
                    sq += v;
                    sqc += v * C[k];
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                sq += __shfl_xor_sync(0xffffffffu, sq, o);
                sqc += __shfl_xor_sync(0xffffffffu, sqc, o);
            }
            const bool on = vc.coupling && sqc > T(0);
            const T zf = on ? sq / sqc : T(0);
#pragma unroll
            for (int k = 0; k < kAniU; ++k) acc[k] += xw * q[k] * ((on && C[k] >= T(0)) ? C[k] * zf : T(1));
        }
    } else {
        T xt = 0;
        for (int wv = 0; wv < nin; ++wv) xt += X[(size_t)wv * g.n_nodes + j];
        const T *wg = a.Wg + (size_t)(j - g.n_atm) * g.ngd;
#pragma unroll
        for (int k = 0; k < kAniU; ++k) {
            const int u = lane + 32 * k;
            acc[k] = u < g.ngd ? Ls[u] + xt * wg[u] : T(0);
        }
    }
    const int nd_j = j < g.n_atm ? g.nd : g.ngd;
#pragma unroll
    for (int k = 0; k < kAniU; ++k) {
        const int u = lane + 32 * k;
        if (u < nd_j) store_halo(a.Lh + (size_t)u * g.npad, g, x, y, z, acc[k]);
    }
}

// Transport: every slot adds rho_i P L(source, direction) to X(i, arrival
// direction).  One block of kAniW warps per group of 128 receiver rows, as
// the edge kernel walks them.
constexpr int kAniW = 4;
template <typename T>
__global__ void __launch_bounds__(32 * kAniW) k_aniso_transport(GridC g, GraphP gp, FieldP<T> f, ViewC vc,
                                                                const T *__restrict__ Pv, const T *__restrict__ Lh,
                                                                T *Xn) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    const T *vrow = Pv + G.vb + 4 * lane;
    for (int t = w; t < G.nt; t += kAniW) {
        const ASlot &d = gp.aslot[G.t0 + t];
        const int4 a0 = __ldg(reinterpret_cast<const int4 *>(&d));
        const int4 a1 = __ldg(reinterpret_cast<const int4 *>(&d) + 1);
        const int src = a0.x, bits = a1.z, dir = a1.w;
        const bool gsrc = (bits >> 11) & 1;
        const int din = gsrc ? g.nd + dir : dir;
        T P[4];
        ld_quad(vrow + (size_t)t * kGroup, P);
        const T *Ld = Lh + (size_t)dir * g.npad;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (G.row[k] < 0 || rho[k] == T(0)) continue;
            const T v = rho[k] * P[k] * __ldg(Ld + G.rp[k] + src);
            if (v != T(0)) atomicAdd(Xn + (size_t)din * g.n_nodes + G.row[k], v);
        }
    }
}

// change of the series term and its size, accumulated in FP64
template <typename T>
__global__ void k_aniso_change(long long n, const T *X, const T *Xn, double *acc) {
    double d2 = 0.0, n2 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = (double)Xn[i], b = (double)X[i];
        d2 += (a - b) * (a - b);
        n2 += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, d2);
        atomicAdd(acc + 1, n2);
    }
}

// x = sum_w X(i, w) into the FP64 haloed vector, and the emission toward the
// instrument E_i = e1_i Theta_i(s0 . v) + sum_w Theta_i(w . v) X(i, w)
template <typename T>
__global__ void k_aniso_finish(GridC g, FieldP<T> f, const T *__restrict__ X, double *x64, T *emis) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_nodes) return;
    const int nin = g.nd + g.ngd;
    const int z = i / g.nxy, r = i - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    double xt = 0.0;
    for (int wv = 0; wv < nin; ++wv) xt += (double)X[(size_t)wv * g.n_nodes + i];
    store_halo(x64, g, x, y, z, xt);
    if (i >= g.n_atm) return;
    T w[MAX_SPECIES];
    T th0 = 0;
    for (int sp = 0; sp < g.S; ++sp) {
        w[sp] = f.wsp[(size_t)sp * g.n_atm + i];
        th0 += w[sp] * f.hg0v[sp];
    }
    T e = 0;
    for (int wv = 0; wv < nin; ++wv) {
        const T xw = X[(size_t)wv * g.n_nodes + i];
        if (xw == T(0)) continue;
        T th = 0;
        for (int sp = 0; sp < g.S; ++sp) th += w[sp] * f.hgv[sp * nin + wv];
        e += th * xw;
    }
    emis[i] = f.e1[i] * th0 + e;
}

template <typename T>
void launch_aniso_prep(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const ViewP &vp, const AniP<T> &a, long long *launches) {
    const int nin = g.nd + g.ngd;
    const long long warps = (long long)g.S * nin * g.nd;
    k_aniso_qcells<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(g, vc, vp, a.Qraw);
    k_aniso_qnorm<T><<<(g.S * nin + 127) / 128, 128, 0, st>>>(g, a.Qraw, a.Q);
    k_aniso_couple<T><<<(g.n_nodes + 127) / 128, 128, 0, st>>>(g, gp, f, vc, a);
    if (launches) *launches += 3;
}

template <typename T>
void launch_aniso_step(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const AniP<T> &a, const T *X, T *Xn, long long *launches) {
    const long long n = (long long)(g.nd + g.ngd) * g.n_nodes;
    k_aniso_leave<T><<<(unsigned)(((long long)g.n_nodes * 32 + 127) / 128), 128, 0, st>>>(g, gp, f, vc, a, X);
    cudaMemsetAsync(Xn, 0, (size_t)n * sizeof(T), st);
    k_aniso_transport<T><<<(g.nz + 1) * g.gpl, 32 * kAniW, 0, st>>>(g, gp, f, vc, f.val, a.Lh, Xn);
    cudaMemsetAsync(a.acc, 0, 2 * sizeof(double), st);
    k_aniso_change<T><<<512, 256, 0, st>>>(n, X, Xn, a.acc);
    if (launches) *launches += 3;
}

template <typename T>
void launch_aniso_finish(cudaStream_t st, const GridC &g, const FieldP<T> &f, const T *X, double *x64, T *emis,
                         long long *launches) {
    k_aniso_finish<T><<<(g.n_nodes + 127) / 128, 128, 0, st>>>(g, f, X, x64, emis);
    if (launches) *launches += 1;
}

#define INST(T)                                                                                                 \
    template void launch_aniso_prep<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,          \
                                       const ViewC &, const ViewP &, const AniP<T> &, long long *);             \
    template void launch_aniso_step<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,          \
                                       const ViewC &, const AniP<T> &, const T *, T *, long long *);            \
    template void launch_aniso_finish<T>(cudaStream_t, const GridC &, const FieldP<T> &, const T *, double *,   \
                                         T *, long long *);
INST(float)
INST(double)
#undef INST

}  // namespace tk
