// Detector radiance (final radiance sum of Sec. 2 of Mikkonen et al.;
// step 5 of the algorithm in Sec. 3): emission of every voxel toward the
// instrument, then a line-of-sight integration per pixel.
//
//   E_i = e1_i Theta_i(s0 . v) + sum_{in-edges (j,u)} Theta_i(u . v)
//                                   (K^sun_{ij,u} e1_j + K_{ij,u} x_j)
//   L_p = sum_{LOS voxels} exp(-tau_in) (1 - exp(-mu_e ds)) / mu_e E_i / V
//         + exp(-tau_total) (e1_c + x_c) / (pi hx hy)
// The K^sun part of E_i is accumulated during assembly (gsun).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kern.h"
#include "stage.cuh"
#include "first_order.h"

namespace tk {

template <typename T>
__device__ __forceinline__ T rexp(T a);
template <>
__device__ __forceinline__ float rexp<float>(float a) { return expf(a); }
template <>
__device__ __forceinline__ double rexp<double>(double a) { return exp(a); }
template <typename T>
__device__ __forceinline__ T rexpm1(T a);
template <>
__device__ __forceinline__ float rexpm1<float>(float a) { return expm1f(a); }
template <>
__device__ __forceinline__ double rexpm1<double>(double a) { return expm1(a); }

__device__ __forceinline__ int rwrap(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// E_i as one pass over the atmospheric rows of K (the same row-group drivers
// as the solver's sweeps).  Theta_i(u . v) = sum_sp w_sp,i hg_sp(u . v) is
// split by species: for each species the row accumulates
// sum_slots hg_sp(slot direction) K_ij x_j, and the row's species weights
// are applied once at the end.  x is gathered from a compute-type copy (xc)
// of the FP64 solution, in the solver's haloed layout.
#ifndef TK_EMIS_TILE
#define TK_EMIS_TILE 1
#endif
template <typename T, int S>
struct OpEmission {
    using A = T;
    static constexpr int NA = 4 * S;
    static constexpr bool kPart = false;
    struct Slot {
        T hv[S];
    };
    struct Pre {
        T w[S];
        T e1, gsun;
    };
    FieldP<T> f;
    const T *xc;
    T *emis;
    int ndir, n_atm;
    static constexpr int kTile = (sizeof(T) == 4 && TK_EMIS_TILE) ? 1 : 0;
    __device__ __forceinline__ const T *gsrc(int) const { return xc; }
    // the slot's phase-function values toward the instrument, per species
    __device__ __forceinline__ Slot slot(const GraphP &gp, int t) const {
        Slot si;
        const int hgd = __ldg(&gp.aslot[t].hgdir);
#pragma unroll
        for (int sp = 0; sp < S; ++sp) si.hv[sp] = f.hgv[sp * ndir + hgd];
        return si;
    }
    __device__ __forceinline__ void acc(A *a, int k, T vx, const Slot &si) const {
#pragma unroll
        for (int sp = 0; sp < S; ++sp) a[sp * 4 + k] += vx * si.hv[sp];
    }
    __device__ __forceinline__ void add(A *a, int k, T v, int j, const Slot &si) const { acc(a, k, v * __ldg(xc + j), si); }
    __device__ __forceinline__ void add_t(A *a, int k, T v, const T *s, int, const Slot &si) const {
        acc(a, k, v * s[0], si);
    }
    __device__ __forceinline__ Pre pre(const GroupRows &G, int k) const {
        Pre p;
        const int i = G.row[k];
#pragma unroll
        for (int sp = 0; sp < S; ++sp) p.w[sp] = f.wsp[(size_t)sp * n_atm + i];
        p.e1 = f.e1[i];
        p.gsun = f.gsun[i];
        return p;
    }
    template <int W>
    __device__ __forceinline__ static void combine_row(const A (*sh)[NA][32], int lane, int k, A *a) {
#pragma unroll
        for (int sp = 0; sp < S; ++sp) sum_word<W, A, NA>(sh, lane, sp * 4 + k, a);
    }
    __device__ __forceinline__ double finish_row(const GroupRows &G, int k, const A *a, const Pre &p) const {
        T tot = T(0), th0 = T(0);
#pragma unroll
        for (int sp = 0; sp < S; ++sp) {
            tot += p.w[sp] * a[sp * 4 + k];
            th0 += p.w[sp] * f.hg0v[sp];
        }
        emis[G.row[k]] = p.e1 * th0 + p.gsun + tot;
        return 0.0;
    }
};

// One warp per pixel.  The line of sight's taps are split into 32 contiguous
// chunks; each lane sums its chunk's optical depth and its chunk's
// contribution as seen from the chunk's top, an exclusive warp scan of the
// chunk depths gives each chunk's attenuation from the TOA, and the warp sum
// of the attenuated contributions is the radiance.
template <typename T>
__global__ void k_pixels(GridC g, FieldP<T> f, ViewC vc, ViewP vp, const T *__restrict__ emis,
                         const double *__restrict__ x, T *rad, T *refl) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (p >= vp.npx * vp.npy) return;
    const T *len;
    if constexpr (sizeof(T) == 4)
        len = (const T *)vp.los_len_f;
    else
        len = (const T *)vp.los_len_d;
    const int cx = vp.pix_cx[p], cy = vp.pix_cy[p], cl = vp.pix_cls[p];
    const int off = vp.los_off[cl], n = vp.los_n[cl];
    const T inv_vol = (T)(1.0 / (g.hx * g.hy * g.hz));
    const int per = (n + 31) / 32;
    const int t0 = min(n, lane * per), t1 = min(n, t0 + per);
    T tau = T(0), L = T(0);
    if (t0 < t1) {
        DTap prev = vp.los_taps[off + t0];
        int xw = rwrap(cx + prev.dx, g.nx), yw = rwrap(cy + prev.dy, g.ny);
        for (int t = t0; t < t1; ++t) {
            DTap tp = vp.los_taps[off + t];
            xw += tp.dx - prev.dx;
            xw = xw < 0 ? xw + g.nx : (xw >= g.nx ? xw - g.nx : xw);
            yw += tp.dy - prev.dy;
            yw = yw < 0 ? yw + g.ny : (yw >= g.ny ? yw - g.ny : yw);
            prev = tp;
            const int idx = (tp.dz * g.ny + yw) * g.nx + xw;
            const T me = f.mu_e[idx], ds = len[off + t];
            const T fr = me > T(0) ? -rexpm1<T>(-me * ds) / me : ds;
            L += rexp<T>(-tau) * fr * emis[idx] * inv_vol;
            tau += me * ds;
        }
    }
    // exclusive scan of the chunk depths (fixed order)
    T incl = tau;
    for (int o = 1; o < 32; o <<= 1) {
        T v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const T before = incl - tau;
    T contrib = rexp<T>(-before) * L;
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
    const T total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) {
        const int c = g.n_atm + cy * g.nx + cx;
        T Lp = contrib + rexp<T>(-total) * (f.e1[c] + (T)x[halo_pos(g, cx, cy, g.nz)]) * (T)(1.0 / (3.14159265358979323846 * g.hx * g.hy));
        rad[p] = Lp;
        if (refl) refl[p] = Lp * (T)(3.14159265358979323846 / (vc.mu0 * vc.f0));
    }
}

template <typename T, int S>
static void run_emission(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const T *xc, T *emis) {
    OpEmission<T, S> op;
    op.f = f;
    op.xc = xc;
    op.emis = emis;
    op.ndir = g.nd + g.ngd;
    op.n_atm = g.n_atm;
    // atmospheric layers only: the ground emits nothing toward the instrument
    GridC ge = g;
    ge.wq = g.wq_em;
    run_op(st, ge, gp, f.val, op, 1);
}

template <typename T>
void launch_emission(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                     const T *xc, T *emis) {
    (void)vc;
    switch (g.S) {  // the species count as a compile-time constant
        case 1: run_emission<T, 1>(st, g, gp, f, xc, emis); break;
        case 2: run_emission<T, 2>(st, g, gp, f, xc, emis); break;
        case 3: run_emission<T, 3>(st, g, gp, f, xc, emis); break;
        default: run_emission<T, 4>(st, g, gp, f, xc, emis); break;
    }
}

template <typename T>
void launch_pixels(cudaStream_t st, const GridC &g, const FieldP<T> &f, const ViewC &vc, const ViewP &vp,
                   const T *emis, const double *x, T *rad, T *refl) {
    long long n = (long long)vp.npx * vp.npy * 32;
    k_pixels<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, f, vc, vp, emis, x, rad, refl);
}

// First scattering order only: E_i = e1_i Theta_i(s0 . v), one thread per
// atmospheric node (the species sum in the order of the full pass).
template <typename T>
__global__ void k_emission_first(GridC g, FieldP<T> f, T *emis) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_atm) return;
    T th0 = T(0);
    for (int sp = 0; sp < g.S; ++sp) th0 += f.wsp[(size_t)sp * g.n_atm + i] * f.hg0v[sp];
    emis[i] = f.e1[i] * th0;
}

template <typename T>
void launch_emission_first(cudaStream_t st, const GridC &g, const FieldP<T> &f, T *emis) {
    k_emission_first<T><<<(g.n_atm + 255) / 256, 256, 0, st>>>(g, f, emis);
}

template void launch_emission_first<float>(cudaStream_t, const GridC &, const FieldP<float> &, float *);
template void launch_emission_first<double>(cudaStream_t, const GridC &, const FieldP<double> &, double *);
template void launch_emission<float>(cudaStream_t, const GridC &, const GraphP &, const FieldP<float> &,
                                     const ViewC &, const float *, float *);
template void launch_emission<double>(cudaStream_t, const GridC &, const GraphP &, const FieldP<double> &,
                                      const ViewC &, const double *, double *);
template void launch_pixels<float>(cudaStream_t, const GridC &, const FieldP<float> &, const ViewC &, const ViewP &,
                                   const float *, const double *, float *, float *);
template void launch_pixels<double>(cudaStream_t, const GridC &, const FieldP<double> &, const ViewC &,
                                    const ViewP &, const double *, const double *, double *, double *);

}  // namespace tk
