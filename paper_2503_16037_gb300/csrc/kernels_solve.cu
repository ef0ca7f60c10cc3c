// Solver kernels for (I - K) x = s (Eq. flux_system of Mikkonen et al.;
// the Neumann / source iteration is the series of Eq. fs_sum).
//
// The CSR SpMV walks rows of receivers.  Every row is padded to a multiple of
// four slots (padding slots have value 0 and point at the row itself), so a
// group of G lanes streams each row with 16-byte loads of values and column
// indices; x is gathered through the cache.  Reductions are deterministic:
// fixed grids, fixed per-block order, and a single-thread final sum.
#include <cuda_runtime.h>

#include <cstdint>

#include "kern.h"

namespace tk {

constexpr int MAX_PART = 1024;

__device__ __forceinline__ void load4(const float *v, int q, float &a, float &b, float &c, float &d) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(v) + q);
    a = t.x;
    b = t.y;
    c = t.z;
    d = t.w;
}
__device__ __forceinline__ void load4(const double *v, int q, double &a, double &b, double &c, double &d) {
    const double2 *p = reinterpret_cast<const double2 *>(v) + 2 * (size_t)q;
    double2 t0 = __ldg(p), t1 = __ldg(p + 1);
    a = t0.x;
    b = t0.y;
    c = t1.x;
    d = t1.y;
}

// sum over the slots of one row by a group of G lanes (gl = lane in group)
template <typename T, typename XT, typename AT, int G>
__device__ __forceinline__ AT row_sum(const GraphP &gp, const T *__restrict__ val, const XT *__restrict__ x, int row,
                                      int gl) {
    const int q0 = __ldg(gp.row_ptr + row) >> 2, q1 = __ldg(gp.row_ptr + row + 1) >> 2;
    const int4 *c4 = reinterpret_cast<const int4 *>(gp.col);
    AT acc = AT(0);
    for (int q = q0 + gl; q < q1; q += G) {
        int4 j = __ldg(c4 + q);
        T v0, v1, v2, v3;
        load4(val, q, v0, v1, v2, v3);
        acc += (AT)v0 * (AT)__ldg(x + j.x);
        acc += (AT)v1 * (AT)__ldg(x + j.y);
        acc += (AT)v2 * (AT)__ldg(x + j.z);
        acc += (AT)v3 * (AT)__ldg(x + j.w);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// MODE 0: y = b + K x (b may be null); MODE 1: y = x - K x
template <typename T, int G, int MODE>
__global__ void __launch_bounds__(256) k_spmv(GridC g, GraphP gp, const T *__restrict__ val, const T *__restrict__ x,
                                              const T *__restrict__ b, T *__restrict__ y) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int row = t / G, gl = t & (G - 1);
    bool live = row < g.n_nodes;
    int r = live ? row : g.n_nodes - 1;
    T acc = row_sum<T, T, T, G>(gp, val, x, r, gl);
    if (live && gl == 0) {
        if (MODE == 0)
            y[row] = (b ? b[row] : T(0)) + acc;
        else
            y[row] = x[row] - acc;
    }
}

template <typename T>
void launch_spmv(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, const T *b, T *y) {
    constexpr int G = sizeof(T) == 4 ? 16 : 16;
    long long th = (long long)g.n_nodes * G;
    k_spmv<T, G, 0><<<(unsigned)((th + 255) / 256), 256, 0, st>>>(g, gp, val, x, b, y);
}

template <typename T>
void launch_imk(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, T *y) {
    constexpr int G = 16;
    long long th = (long long)g.n_nodes * G;
    k_spmv<T, G, 1><<<(unsigned)((th + 255) / 256), 256, 0, st>>>(g, gp, val, x, nullptr, y);
}

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

// r = s - x + K x with FP64 x and FP64 accumulation; block partials of r^2
template <typename T, int G>
__global__ void __launch_bounds__(256) k_resid64(GridC g, GraphP gp, const T *__restrict__ val,
                                                 const T *__restrict__ s, const double *__restrict__ x,
                                                 double *__restrict__ r, double *__restrict__ part) {
    const int groups_per_block = blockDim.x / G;
    const int gid = threadIdx.x / G, gl = threadIdx.x & (G - 1);
    const int total = gridDim.x * groups_per_block;
    double loc = 0.0;
    const int n_iter = (g.n_nodes + total - 1) / total;
    for (int it = 0; it < n_iter; ++it) {
        int row = it * total + blockIdx.x * groups_per_block + gid;
        bool live = row < g.n_nodes;
        int rr = live ? row : g.n_nodes - 1;
        double acc = row_sum<T, double, double, G>(gp, val, x, rr, gl);
        if (live && gl == 0) {
            double v = (double)s[row] - x[row] + acc;
            r[row] = v;
            loc += v * v;
        }
    }
    double b = block_sum(loc);
    if (threadIdx.x == 0) part[blockIdx.x] = b;
}

int resid_blocks(const GridC &g) {
    long long groups = (long long)g.n_nodes;
    long long blocks = (groups * 16 + 255) / 256;
    if (blocks > 152 * 4) blocks = 152 * 4;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <typename T>
void launch_resid64(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *s, const double *x,
                    double *r, double *part, int nblk) {
    k_resid64<T, 16><<<nblk, 256, 0, st>>>(g, gp, val, s, x, r, part);
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

__global__ void k_finalize(const double *__restrict__ part, int nblk, int ncol, double *__restrict__ out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncol) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)k * nblk + b];
    out[k] = s;
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
    k_finalize<<<(ncol + 63) / 64, 64, 0, st>>>(part, nblk, ncol, out);
}

template <typename T>
void launch_sumsq(cudaStream_t st, int n, const T *x, double *part, int nblk, double *out) {
    launch_dots<T, T>(st, n, x, 0, 1, x, part, nblk, out);
}

void launch_finalize(cudaStream_t st, const double *part, int nblk, double *out) {
    k_finalize<<<1, 64, 0, st>>>(part, nblk, 1, out);
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
    template void launch_axpby<T>(cudaStream_t, int, double, const T *, double, const T *, T *);
INST(float)
INST(double)
#undef INST
template void launch_convert<double, float>(cudaStream_t, int, const double *, float *);
template void launch_convert<float, double>(cudaStream_t, int, const float *, double *);
template void launch_convert<double, double>(cudaStream_t, int, const double *, double *);
template void launch_convert<float, float>(cudaStream_t, int, const float *, float *);

}  // namespace tk
