// Solver kernels for (I - K) x = s (Eq. flux_system of Mikkonen et al.;
// the Neumann / source iteration is the series of Eq. fs_sum).
//
// The SpMV walks rows of receivers (K in CSR order by row), one thread per
// row; the column of each slot comes from the row template of the row's
// layer instead of a stored index, so only the 4-byte values stream (and stay
// resident in L2 across the sweeps of a solve).  Reductions are
// deterministic: fixed grids, fixed per-block order, fixed-order trees.
#include <cuda_runtime.h>

#include <cstdint>

#include "kern.h"

namespace tk {

// Rows are processed in groups of 32 consecutive rows (one per lane) by
// kSplit warps; warp w sums the slots t = w, w + kSplit, ... of its lane's
// row.  The value loads of a warp are coalesced (a slot's values are
// contiguous across the rows of a layer), the x gathers of consecutive rows
// hit consecutive entries (apart from the periodic wrap), and the partial
// sums are combined in shared memory in a fixed order.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    }
    return r;  // valid in thread 0
}

constexpr int kSplit = 4;

template <typename T, typename XT, typename AT>
__device__ __forceinline__ AT row_part(const GridC &g, const GraphP &gp, const T *__restrict__ val,
                                       const XT *__restrict__ x, int row, int w) {
    const int z = row / g.nxy, r = row - z * g.nxy, yy = r / g.nx, xx = r - yy * g.nx;
    const int t0 = __ldg(gp.tstart + z), nt = __ldg(gp.tstart + z + 1) - t0;
    const T *v = val + val_base(__ldg(gp.voff + z), nt, r);
    const size_t stride = (size_t)kGroup;
    AT acc = AT(0);
#pragma unroll 4
    for (int t = w; t < nt; t += kSplit) {
        const int4 te = __ldg(gp.tmpl + t0 + t);
        const int j = slot_src(g, row, xx, yy, te);
        acc += (AT)__ldg(v + (size_t)t * stride) * (AT)__ldg(x + j);
    }
    return acc;
}

// combine the kSplit partial sums of each row; valid in warp 0
template <typename AT>
__device__ __forceinline__ AT combine_parts(AT part) {
    __shared__ AT sh[kSplit][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    sh[w][lane] = part;
    __syncthreads();
    AT tot = AT(0);
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < kSplit; ++k) tot += sh[k][lane];
    }
    return tot;
}

// ---- four rows per thread (nx divisible by 4): rows row0 .. row0 + 3 share y
// and the template, their values of a slot are one aligned 16-byte load, and
// their sources are consecutive apart from the periodic wrap in x.
constexpr int kQSplit = 8;

template <typename T>
struct Vec4T;
template <>
struct Vec4T<float> {
    __device__ static __forceinline__ void load(const float *p, float &a, float &b, float &c, float &d) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        a = v.x;
        b = v.y;
        c = v.z;
        d = v.w;
    }
};
template <>
struct Vec4T<double> {
    __device__ static __forceinline__ void load(const double *p, double &a, double &b, double &c, double &d) {
        double2 v0 = __ldg(reinterpret_cast<const double2 *>(p)), v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        a = v0.x;
        b = v0.y;
        c = v1.x;
        d = v1.y;
    }
};

template <typename T, typename XT, typename AT>
__device__ __forceinline__ void quad_part(const GridC &g, const GraphP &gp, const T *__restrict__ val,
                                          const XT *__restrict__ x, int row0, int w, AT acc[4]) {
    const int z = row0 / g.nxy, r0 = row0 - z * g.nxy, y = r0 / g.nx, x0 = r0 - y * g.nx;
    const int t0 = __ldg(gp.tstart + z), nt = __ldg(gp.tstart + z + 1) - t0;
    const T *v = val + val_base(__ldg(gp.voff + z), nt, r0);
    const size_t stride = (size_t)kGroup;
#pragma unroll 2
    for (int t = w; t < nt; t += kQSplit) {
        const int4 te = __ldg(gp.tmpl + t0 + t);
        const int sy = y + tmpl_sdy(te), sx = x0 + tmpl_sdx(te);
        const int jb = row0 + te.y + (sy < 0 ? g.nxy : 0) - (sy >= g.ny ? g.nxy : 0);
        T v0, v1, v2, v3;
        Vec4T<T>::load(v + (size_t)t * stride, v0, v1, v2, v3);
        const int j0 = jb + (sx < 0 ? g.nx : 0) - (sx >= g.nx ? g.nx : 0);
        const int j1 = jb + 1 + (sx + 1 < 0 ? g.nx : 0) - (sx + 1 >= g.nx ? g.nx : 0);
        const int j2 = jb + 2 + (sx + 2 < 0 ? g.nx : 0) - (sx + 2 >= g.nx ? g.nx : 0);
        const int j3 = jb + 3 + (sx + 3 < 0 ? g.nx : 0) - (sx + 3 >= g.nx ? g.nx : 0);
        acc[0] += (AT)v0 * (AT)__ldg(x + j0);
        acc[1] += (AT)v1 * (AT)__ldg(x + j1);
        acc[2] += (AT)v2 * (AT)__ldg(x + j2);
        acc[3] += (AT)v3 * (AT)__ldg(x + j3);
    }
}

// combine kQSplit partials of four rows per lane; valid in warp 0
template <typename AT>
__device__ __forceinline__ void combine_quad(AT acc[4]) {
    __shared__ AT sh[kQSplit][4][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; ++k) sh[w][k][lane] = acc[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            AT t = AT(0);
#pragma unroll
            for (int q = 0; q < kQSplit; ++q) t += sh[q][k][lane];
            acc[k] = t;
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(32 * kQSplit) k_spmv4(GridC g, GraphP gp, const T *__restrict__ val,
                                                        const T *__restrict__ x, const T *__restrict__ b,
                                                        T *__restrict__ y) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = (blockIdx.x * 32 + lane) * 4;
    const bool live = row0 < g.n_nodes;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    if (live) quad_part<T, T, T>(g, gp, val, x, row0, w, acc);
    combine_quad<T>(acc);
    if (w == 0 && live) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (MODE == 0)
                y[row0 + k] = (b ? b[row0 + k] : T(0)) + acc[k];
            else
                y[row0 + k] = x[row0 + k] - acc[k];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * kQSplit) k_resid64_4(GridC g, GraphP gp, const T *__restrict__ val,
                                                            const T *__restrict__ s, const double *__restrict__ x,
                                                            double *__restrict__ r, double *__restrict__ part) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = (blockIdx.x * 32 + lane) * 4;
    const bool live = row0 < g.n_nodes;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (live) quad_part<T, double, double>(g, gp, val, x, row0, w, acc);
    combine_quad<double>(acc);
    double sq = 0.0;
    if (w == 0 && live) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double v = (double)s[row0 + k] - x[row0 + k] + acc[k];
            r[row0 + k] = v;
            sq += v * v;
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) red[w] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kQSplit; ++i) t += red[i];
        part[blockIdx.x] = t;
    }
}

// Neumann sweep that also records ||y - x||^2 per block (the norm of K^k r
// along the series, for the power estimate of the largest eigenvalue)
template <typename T>
__global__ void __launch_bounds__(32 * kQSplit) k_sweep_pow4(GridC g, GraphP gp, const T *__restrict__ val,
                                                             const T *__restrict__ x, const T *__restrict__ b,
                                                             T *__restrict__ y, double *__restrict__ part) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = (blockIdx.x * 32 + lane) * 4;
    const bool live = row0 < g.n_nodes;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    if (live) quad_part<T, T, T>(g, gp, val, x, row0, w, acc);
    combine_quad<T>(acc);
    double sq = 0.0;
    if (w == 0 && live) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            T v = b[row0 + k] + acc[k];
            double dd = (double)v - (double)x[row0 + k];
            sq += dd * dd;
            y[row0 + k] = v;
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) red[w] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kQSplit; ++i) t += red[i];
        part[blockIdx.x] = t;
    }
}

// One Chebyshev step on (I - K) d = r0 (three-term form):
//   q = K p;  r <- r - p + q;  d <- d + p;  p' = c1 p + c2 r
template <typename T>
__global__ void __launch_bounds__(32 * kQSplit) k_cheb4(GridC g, GraphP gp, const T *__restrict__ val,
                                                        const T *__restrict__ p, T *__restrict__ r,
                                                        T *__restrict__ d, T *__restrict__ pn, T c1, T c2) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = (blockIdx.x * 32 + lane) * 4;
    const bool live = row0 < g.n_nodes;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    if (live) quad_part<T, T, T>(g, gp, val, p, row0, w, acc);
    combine_quad<T>(acc);
    if (w == 0 && live) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = row0 + k;
            const T pi = p[i];
            const T rr = r[i] - pi + acc[k];
            r[i] = rr;
            d[i] += pi;
            pn[i] = c1 * pi + c2 * rr;
        }
    }
}

// ---- residual in double-single arithmetic (pairs of FP32 numbers).  x is
// held as x_hi + x_lo (x_hi = fl32(x), x_lo = fl32(x - x_hi)); each product
// v x_hi is split exactly into p + e with an FMA (two-product), the p are
// summed with Knuth's two-sum and all low-order parts are gathered in a
// second FP32 accumulator.  The row sum so obtained carries a relative error
// of order 2^-48 per term instead of 2^-24.
// (explicitly rounded operations: none of them may be contracted into an FMA)
__device__ __forceinline__ void ds_add_prod(float &hi, float &lo, float v, float xh, float xl) {
    const float p = __fmul_rn(v, xh);
    const float e = fmaf(v, xh, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(err, e), __fmul_rn(v, xl)));
}

__device__ __forceinline__ void quad_part_ds(const GridC &g, const GraphP &gp, const float *__restrict__ val,
                                             const float *__restrict__ xh, const float *__restrict__ xl, int row0,
                                             int w, double acc[4]) {
    const int z = row0 / g.nxy, r0 = row0 - z * g.nxy, y = r0 / g.nx, x0 = r0 - y * g.nx;
    const int t0 = __ldg(gp.tstart + z), nt = __ldg(gp.tstart + z + 1) - t0;
    const float *v = val + val_base(__ldg(gp.voff + z), nt, r0);
    float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f, l3 = 0.f;
#pragma unroll 2
    for (int t = w; t < nt; t += kQSplit) {
        const int4 te = __ldg(gp.tmpl + t0 + t);
        const int sy = y + tmpl_sdy(te), sx = x0 + tmpl_sdx(te);
        const int jb = row0 + te.y + (sy < 0 ? g.nxy : 0) - (sy >= g.ny ? g.nxy : 0);
        float v0, v1, v2, v3;
        Vec4T<float>::load(v + (size_t)t * kGroup, v0, v1, v2, v3);
        const int j0 = jb + (sx < 0 ? g.nx : 0) - (sx >= g.nx ? g.nx : 0);
        const int j1 = jb + 1 + (sx + 1 < 0 ? g.nx : 0) - (sx + 1 >= g.nx ? g.nx : 0);
        const int j2 = jb + 2 + (sx + 2 < 0 ? g.nx : 0) - (sx + 2 >= g.nx ? g.nx : 0);
        const int j3 = jb + 3 + (sx + 3 < 0 ? g.nx : 0) - (sx + 3 >= g.nx ? g.nx : 0);
        ds_add_prod(h0, l0, v0, __ldg(xh + j0), __ldg(xl + j0));
        ds_add_prod(h1, l1, v1, __ldg(xh + j1), __ldg(xl + j1));
        ds_add_prod(h2, l2, v2, __ldg(xh + j2), __ldg(xl + j2));
        ds_add_prod(h3, l3, v3, __ldg(xh + j3), __ldg(xl + j3));
    }
    acc[0] = (double)h0 + (double)l0;
    acc[1] = (double)h1 + (double)l1;
    acc[2] = (double)h2 + (double)l2;
    acc[3] = (double)h3 + (double)l3;
}

__global__ void __launch_bounds__(32 * kQSplit) k_resid_ds4(GridC g, GraphP gp, const float *__restrict__ val,
                                                            const float *__restrict__ s, const double *__restrict__ x,
                                                            const float *__restrict__ xh,
                                                            const float *__restrict__ xl, double *__restrict__ r,
                                                            double *__restrict__ part) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = (blockIdx.x * 32 + lane) * 4;
    const bool live = row0 < g.n_nodes;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (live) quad_part_ds(g, gp, val, xh, xl, row0, w, acc);
    combine_quad<double>(acc);
    double sq = 0.0;
    if (w == 0 && live) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double vv = (double)s[row0 + k] - x[row0 + k] + acc[k];
            r[row0 + k] = vv;
            sq += vv * vv;
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) red[w] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kQSplit; ++i) t += red[i];
        part[blockIdx.x] = t;
    }
}

// x += d, with the double-single split of the new x
template <typename T>
__global__ void k_update_x(int n, const T *__restrict__ d, double *__restrict__ x, float *__restrict__ xh,
                           float *__restrict__ xl) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = x[i] + (double)d[i];
    x[i] = v;
    if (xh) {
        float h = (float)v;
        xh[i] = h;
        xl[i] = (float)(v - (double)h);
    }
}

static bool quad_ok(const GridC &g) { return g.nx % 4 == 0; }

// MODE 0: y = b + K x (b may be null); MODE 1: y = x - K x
template <typename T, int MODE>
__global__ void __launch_bounds__(32 * kSplit) k_spmv(GridC g, GraphP gp, const T *__restrict__ val,
                                                      const T *__restrict__ x, const T *__restrict__ b,
                                                      T *__restrict__ y) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 32 + lane;
    const bool live = row < g.n_nodes;
    T part = live ? row_part<T, T, T>(g, gp, val, x, row, w) : T(0);
    T acc = combine_parts<T>(part);
    if (w == 0 && live) {
        if (MODE == 0)
            y[row] = (b ? b[row] : T(0)) + acc;
        else
            y[row] = x[row] - acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * kSplit) k_sweep_pow(GridC g, GraphP gp, const T *__restrict__ val,
                                                           const T *__restrict__ x, const T *__restrict__ b,
                                                           T *__restrict__ y, double *__restrict__ part) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 32 + lane;
    const bool live = row < g.n_nodes;
    T pr = live ? row_part<T, T, T>(g, gp, val, x, row, w) : T(0);
    T acc = combine_parts<T>(pr);
    double sq = 0.0;
    if (w == 0 && live) {
        T v = b[row] + acc;
        double dd = (double)v - (double)x[row];
        sq = dd * dd;
        y[row] = v;
    }
    double bs = block_sum(sq);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
}

template <typename T>
__global__ void __launch_bounds__(32 * kSplit) k_cheb(GridC g, GraphP gp, const T *__restrict__ val,
                                                      const T *__restrict__ p, T *__restrict__ r, T *__restrict__ d,
                                                      T *__restrict__ pn, T c1, T c2) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 32 + lane;
    const bool live = row < g.n_nodes;
    T pr = live ? row_part<T, T, T>(g, gp, val, p, row, w) : T(0);
    T acc = combine_parts<T>(pr);
    if (w == 0 && live) {
        const T pi = p[row];
        const T rr = r[row] - pi + acc;
        r[row] = rr;
        d[row] += pi;
        pn[row] = c1 * pi + c2 * rr;
    }
}

int sweep_blocks(const GridC &g) { return quad_ok(g) ? (g.n_nodes / 4 + 31) / 32 : (g.n_nodes + 31) / 32; }

template <typename T>
void launch_sweep_pow(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, const T *b, T *y,
                      double *part) {
    if (quad_ok(g))
        k_sweep_pow4<T><<<sweep_blocks(g), 32 * kQSplit, 0, st>>>(g, gp, val, x, b, y, part);
    else
        k_sweep_pow<T><<<sweep_blocks(g), 32 * kSplit, 0, st>>>(g, gp, val, x, b, y, part);
}

template <typename T>
void launch_cheb(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *p, T *r, T *d, T *pn,
                 double c1, double c2) {
    if (quad_ok(g))
        k_cheb4<T><<<sweep_blocks(g), 32 * kQSplit, 0, st>>>(g, gp, val, p, r, d, pn, (T)c1, (T)c2);
    else
        k_cheb<T><<<sweep_blocks(g), 32 * kSplit, 0, st>>>(g, gp, val, p, r, d, pn, (T)c1, (T)c2);
}

template <typename T>
void launch_spmv(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, const T *b, T *y) {
    if (quad_ok(g))
        k_spmv4<T, 0><<<(g.n_nodes / 4 + 31) / 32, 32 * kQSplit, 0, st>>>(g, gp, val, x, b, y);
    else
        k_spmv<T, 0><<<(g.n_nodes + 31) / 32, 32 * kSplit, 0, st>>>(g, gp, val, x, b, y);
}

template <typename T>
void launch_imk(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, T *y) {
    if (quad_ok(g))
        k_spmv4<T, 1><<<(g.n_nodes / 4 + 31) / 32, 32 * kQSplit, 0, st>>>(g, gp, val, x, nullptr, y);
    else
        k_spmv<T, 1><<<(g.n_nodes + 31) / 32, 32 * kSplit, 0, st>>>(g, gp, val, x, nullptr, y);
}


// r = s - x + K x with FP64 x and FP64 accumulation; per-block sums of r^2
template <typename T>
__global__ void __launch_bounds__(32 * kSplit) k_resid64(GridC g, GraphP gp, const T *__restrict__ val,
                                                         const T *__restrict__ s, const double *__restrict__ x,
                                                         double *__restrict__ r, double *__restrict__ part) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 32 + lane;
    const bool live = row < g.n_nodes;
    double p = live ? row_part<T, double, double>(g, gp, val, x, row, w) : 0.0;
    double acc = combine_parts<double>(p);
    double sq = 0.0;
    if (w == 0 && live) {
        double v = (double)s[row] - x[row] + acc;
        r[row] = v;
        sq = v * v;
    }
    double b = block_sum(sq);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
}

int resid_blocks(const GridC &g) { return quad_ok(g) ? (g.n_nodes / 4 + 31) / 32 : (g.n_nodes + 31) / 32; }

bool resid_ds_ok(const GridC &g) { return quad_ok(g); }

void launch_resid_ds(cudaStream_t st, const GridC &g, const GraphP &gp, const float *val, const float *s,
                     const double *x, const float *xh, const float *xl, double *r, double *part, int nblk) {
    k_resid_ds4<<<nblk, 32 * kQSplit, 0, st>>>(g, gp, val, s, x, xh, xl, r, part);
}

template <typename T>
void launch_update_x(cudaStream_t st, int n, const T *d, double *x, float *xh, float *xl) {
    k_update_x<T><<<(n + 255) / 256, 256, 0, st>>>(n, d, x, xh, xl);
}

template <typename T>
void launch_resid64(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *s, const double *x,
                    double *r, double *part, int nblk) {
    if (quad_ok(g))
        k_resid64_4<T><<<nblk, 32 * kQSplit, 0, st>>>(g, gp, val, s, x, r, part);
    else
        k_resid64<T><<<nblk, 32 * kSplit, 0, st>>>(g, gp, val, s, x, r, part);
}

// ---------------------------------------------------------------------------
// Reductions

template <typename A, typename B>
__global__ void k_dots(int n, const A *__restrict__ V, size_t ldv, int ncol, const B *__restrict__ y,
                       double *__restrict__ part) {
    for (int k = 0; k < ncol; ++k) {
        const A *v = V + (size_t)k * ldv;
        double acc = 0.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
            acc += (double)v[i] * (double)y[i];
        double b = block_sum(acc);
        if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = b;
    }
}

// one block per column; fixed strided partial sums then a fixed-order tree
__global__ void k_finalize(const double *__restrict__ part, int nblk, int ncol, double *__restrict__ out) {
    __shared__ double sh[256];
    int k = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(size_t)k * nblk + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
    (void)ncol;
}

int dot_blocks(int n) {
    long long b = ((long long)n + 2047) / 2048;
    if (b > 296) b = 296;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename A, typename B>
void launch_dots(cudaStream_t st, int n, const A *V, size_t ldv, int ncol, const B *y, double *part, int nblk,
                 double *out) {
    k_dots<A, B><<<nblk, 256, 0, st>>>(n, V, ldv, ncol, y, part);
    k_finalize<<<ncol, 256, 0, st>>>(part, nblk, ncol, out);
}

template <typename T>
void launch_sumsq(cudaStream_t st, int n, const T *x, double *part, int nblk, double *out) {
    launch_dots<T, T>(st, n, x, 0, 1, x, part, nblk, out);
}

void launch_finalize2(cudaStream_t st, const double *part, int nblk, double *out) {
    k_finalize<<<2, 256, 0, st>>>(part, nblk, 2, out);
}

void launch_finalize(cudaStream_t st, const double *part, int nblk, double *out) {
    k_finalize<<<1, 256, 0, st>>>(part, nblk, 1, out);
}

// ---------------------------------------------------------------------------
// Vector operations

template <typename T, typename U>
__global__ void k_convert(int n, const T *__restrict__ a, U *__restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (U)a[i];
}
template <typename T>
__global__ void k_axpy64(int n, const T *__restrict__ d, double *__restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += (double)d[i];
}
template <typename T>
__global__ void k_scale(int n, const T *__restrict__ a, double alpha, T *__restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (T)(alpha * (double)a[i]);
}
template <typename T>
__global__ void k_gupdate(int n, T *__restrict__ w, const T *__restrict__ V, size_t ldv, int k,
                          const double *__restrict__ h, double sign) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = (double)w[i];
    for (int j = 0; j < k; ++j) acc += sign * h[j] * (double)V[(size_t)j * ldv + i];
    w[i] = (T)acc;
}

template <typename T, typename U>
void launch_convert(cudaStream_t st, int n, const T *a, U *b) {
    k_convert<T, U><<<(n + 255) / 256, 256, 0, st>>>(n, a, b);
}
template <typename T>
void launch_axpy_to64(cudaStream_t st, int n, const T *d, double *x) {
    k_axpy64<T><<<(n + 255) / 256, 256, 0, st>>>(n, d, x);
}
template <typename T>
void launch_scale(cudaStream_t st, int n, const T *a, double alpha, T *b) {
    k_scale<T><<<(n + 255) / 256, 256, 0, st>>>(n, a, alpha, b);
}
template <typename T>
void launch_gmres_update(cudaStream_t st, int n, T *w, const T *V, size_t ldv, int k, const double *h) {
    k_gupdate<T><<<(n + 255) / 256, 256, 0, st>>>(n, w, V, ldv, k, h, -1.0);
}
template <typename T>
void launch_combine(cudaStream_t st, int n, T *x, const T *V, size_t ldv, int k, const double *y) {
    k_gupdate<T><<<(n + 255) / 256, 256, 0, st>>>(n, x, V, ldv, k, y, 1.0);
}

template <typename T>
__global__ void k_axpby(int n, double a, const T *__restrict__ x, double b, const T *__restrict__ y,
                        T *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (T)(a * (double)x[i] + b * (double)y[i]);
}
template <typename T>
void launch_axpby(cudaStream_t st, int n, double a, const T *x, double b, const T *y, T *out) {
    k_axpby<T><<<(n + 255) / 256, 256, 0, st>>>(n, a, x, b, y, out);
}

#define INST(T)                                                                                                    \
    template void launch_spmv<T>(cudaStream_t, const GridC &, const GraphP &, const T *, const T *, const T *, T *); \
    template void launch_imk<T>(cudaStream_t, const GridC &, const GraphP &, const T *, const T *, T *);             \
    template void launch_resid64<T>(cudaStream_t, const GridC &, const GraphP &, const T *, const T *,               \
                                    const double *, double *, double *, int);                                       \
    template void launch_dots<T, T>(cudaStream_t, int, const T *, size_t, int, const T *, double *, int, double *); \
    template void launch_sumsq<T>(cudaStream_t, int, const T *, double *, int, double *);                           \
    template void launch_axpy_to64<T>(cudaStream_t, int, const T *, double *);                                      \
    template void launch_scale<T>(cudaStream_t, int, const T *, double, T *);                                       \
    template void launch_gmres_update<T>(cudaStream_t, int, T *, const T *, size_t, int, const double *);           \
    template void launch_combine<T>(cudaStream_t, int, T *, const T *, size_t, int, const double *);            \
    template void launch_axpby<T>(cudaStream_t, int, double, const T *, double, const T *, T *);                   \
    template void launch_update_x<T>(cudaStream_t, int, const T *, double *, float *, float *);                   \
    template void launch_sweep_pow<T>(cudaStream_t, const GridC &, const GraphP &, const T *, const T *,          \
                                      const T *, T *, double *);                                                \
    template void launch_cheb<T>(cudaStream_t, const GridC &, const GraphP &, const T *, const T *, T *, T *,     \
                                 T *, double, double);
INST(float)
INST(double)
#undef INST
template void launch_convert<double, float>(cudaStream_t, int, const double *, float *);
template void launch_convert<float, double>(cudaStream_t, int, const float *, double *);
template void launch_convert<double, double>(cudaStream_t, int, const double *, double *);
template void launch_convert<float, float>(cudaStream_t, int, const float *, float *);

}  // namespace tk
