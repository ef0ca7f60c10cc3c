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

// Rows in groups of 32 (one per lane) shared by kEmSplit warps, each summing
// every kEmSplit-th slot of the template; partials combined in a fixed order.
constexpr int kEmSplit = 4;

template <typename T>
__global__ void __launch_bounds__(32 * kEmSplit) k_emission(GridC g, GraphP gp, FieldP<T> f, ViewC vc,
                                                            const double *x, T *emis) {
    __shared__ T sh[kEmSplit][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 32 + lane;
    const bool live = row < g.n_atm;
    const int ndir = g.nd + g.ngd;
    T acc = T(0);
    T wr[MAX_SPECIES];
    if (live) {
        const int z = row / g.nxy, r = row - z * g.nxy, yy = r / g.nx, xx = r - yy * g.nx;
        const int t0 = gp.tstart[z], nt = gp.tstart[z + 1] - t0;
        const T *v = f.val + val_base(gp.voff[z], nt, r);
        for (int sp = 0; sp < g.S; ++sp) wr[sp] = f.wsp[(size_t)sp * g.n_atm + row];
        for (int t = w; t < nt; t += kEmSplit) {
            const int4 te = __ldg(gp.tmpl + t0 + t);
            const int hgd = gp.cls[te.x].hgdir;
            T th = T(0);
            for (int sp = 0; sp < g.S; ++sp) th += wr[sp] * f.hgv[sp * ndir + hgd];
            const int j = slot_src(g, row, xx, yy, te);
            acc += th * v[(size_t)t * kGroup] * (T)x[j];
        }
    }
    sh[w][lane] = acc;
    __syncthreads();
    if (w == 0 && live) {
        T tot = T(0);
        for (int k = 0; k < kEmSplit; ++k) tot += sh[k][lane];
        T th0 = T(0);
        for (int sp = 0; sp < g.S; ++sp) th0 += wr[sp] * f.hg0v[sp];
        emis[row] = f.e1[row] * th0 + f.gsun[row] + tot;
    }
}

template <typename T>
__global__ void k_pixels(GridC g, FieldP<T> f, ViewC vc, ViewP vp, const T *__restrict__ emis,
                         const double *__restrict__ x, T *rad, T *refl) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= vp.npx * vp.npy) return;
    const T *len;
    if constexpr (sizeof(T) == 4)
        len = (const T *)vp.los_len_f;
    else
        len = (const T *)vp.los_len_d;
    int cx = vp.pix_cx[p], cy = vp.pix_cy[p], cl = vp.pix_cls[p];
    int off = vp.los_off[cl], n = vp.los_n[cl];
    const T inv_vol = (T)(1.0 / (g.hx * g.hy * g.hz));
    T tau = T(0), L = T(0);
    if (n > 0) {
        // taps run along the ray: wrap the first column once, then follow it
        DTap prev = vp.los_taps[off];
        int xw = rwrap(cx + prev.dx, g.nx), yw = rwrap(cy + prev.dy, g.ny);
        for (int t = 0; t < n; ++t) {
            DTap tp = vp.los_taps[off + t];
            xw += tp.dx - prev.dx;
            xw = xw < 0 ? xw + g.nx : (xw >= g.nx ? xw - g.nx : xw);
            yw += tp.dy - prev.dy;
            yw = yw < 0 ? yw + g.ny : (yw >= g.ny ? yw - g.ny : yw);
            prev = tp;
            int idx = (tp.dz * g.ny + yw) * g.nx + xw;
            T me = f.mu_e[idx], ds = len[off + t];
            T fr = me > T(0) ? -rexpm1<T>(-me * ds) / me : ds;
            L += rexp<T>(-tau) * fr * emis[idx] * inv_vol;
            tau += me * ds;
        }
    }
    int c = g.n_atm + cy * g.nx + cx;
    L += rexp<T>(-tau) * (f.e1[c] + (T)x[c]) * (T)(1.0 / (3.14159265358979323846 * g.hx * g.hy));
    rad[p] = L;
    if (refl) refl[p] = L * (T)(3.14159265358979323846 / (vc.mu0 * vc.f0));
}

template <typename T>
void launch_emission(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                     const double *x, T *emis) {
    k_emission<T><<<(g.n_atm + 31) / 32, 32 * kEmSplit, 0, st>>>(g, gp, f, vc, x, emis);
}

template <typename T>
void launch_pixels(cudaStream_t st, const GridC &g, const FieldP<T> &f, const ViewC &vc, const ViewP &vp,
                   const T *emis, const double *x, T *rad, T *refl) {
    int n = vp.npx * vp.npy;
    k_pixels<T><<<(n + 127) / 128, 128, 0, st>>>(g, f, vc, vp, emis, x, rad, refl);
}

template void launch_emission<float>(cudaStream_t, const GridC &, const GraphP &, const FieldP<float> &,
                                     const ViewC &, const double *, float *);
template void launch_emission<double>(cudaStream_t, const GridC &, const GraphP &, const FieldP<double> &,
                                      const ViewC &, const double *, double *);
template void launch_pixels<float>(cudaStream_t, const GridC &, const FieldP<float> &, const ViewC &, const ViewP &,
                                   const float *, const double *, float *, float *);
template void launch_pixels<double>(cudaStream_t, const GridC &, const FieldP<double> &, const ViewC &,
                                    const ViewP &, const double *, const double *, double *, double *);

}  // namespace tk
