// Device helpers of the edge march, shared by the forward edge kernels and
// their adjoint.
#pragma once
#include <cuda_runtime.h>

#include "kern.h"

namespace tk {

template <typename T>
__device__ __forceinline__ T dexp(T a);
template <>
__device__ __forceinline__ float dexp<float>(float a) { return expf(a); }
template <>
__device__ __forceinline__ double dexp<double>(double a) { return exp(a); }
template <typename T>
__device__ __forceinline__ T dexpm1(T a);
template <>
__device__ __forceinline__ float dexpm1<float>(float a) { return expm1f(a); }
template <>
__device__ __forceinline__ double dexpm1<double>(double a) { return expm1(a); }
template <typename T>
__device__ __forceinline__ T dsqrt(T a);
template <>
__device__ __forceinline__ float dsqrt<float>(float a) { return sqrtf(a); }
template <>
__device__ __forceinline__ double dsqrt<double>(double a) { return sqrt(a); }

// 1 - exp(-t) for t >= 0 in the edge kernel.  FP32: the Taylor series
// t - t^2/2 + ... - t^8/8! below t = 1/4 (truncation below 2e-9 relative),
// 1 - __expf(-t) above it (cancellation there is at most a factor 4.6);
// FP64: expm1.
template <typename T>
__device__ __forceinline__ T one_minus_exp(T t);
template <>
__device__ __forceinline__ float one_minus_exp<float>(float t) {
    if (t < 0.25f) {
        float p = 1.f - t * (1.f / 8.f);
        p = 1.f - t * (1.f / 7.f) * p;
        p = 1.f - t * (1.f / 6.f) * p;
        p = 1.f - t * (1.f / 5.f) * p;
        p = 1.f - t * (1.f / 4.f) * p;
        p = 1.f - t * (1.f / 3.f) * p;
        p = 1.f - t * (1.f / 2.f) * p;
        return t * p;
    }
    return 1.f - __expf(-t);
}
template <>
__device__ __forceinline__ double one_minus_exp<double>(double t) { return -expm1(-t); }
template <typename T>
__device__ __forceinline__ T fast_exp_neg(T t);
template <>
__device__ __forceinline__ float fast_exp_neg<float>(float t) { return __expf(-t); }
template <>
__device__ __forceinline__ double fast_exp_neg<double>(double t) { return exp(-t); }

template <typename T>
__device__ __forceinline__ const T *tap_len(const GraphP &gp);
template <>
__device__ __forceinline__ const float *tap_len<float>(const GraphP &gp) { return gp.tap_len_f; }
template <>
__device__ __forceinline__ const double *tap_len<double>(const GraphP &gp) { return gp.tap_len_d; }

__device__ __forceinline__ int wrap_small(int a, int n) {  // -n <= a < 2n
    a = a < 0 ? a + n : a;
    return a >= n ? a - n : a;
}
__device__ __forceinline__ int wrap_any(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// optical depth of a stencil-sized tap list based at cell (bx, by, bz)
template <typename T>
__device__ __forceinline__ T tap_sum(const GridC &g, const GraphP &gp, const T *__restrict__ mu_e, int off, int n,
                                     int bx, int by, int bz) {
    const T *len = tap_len<T>(gp);
    T acc = T(0);
    for (int t = 0; t < n; ++t) {
        DTap tp = gp.taps[off + t];
        int x = wrap_small(bx + tp.dx, g.nx), y = wrap_small(by + tp.dy, g.ny), z = bz + tp.dz;
        acc += len[off + t] * __ldg(mu_e + (z * g.ny + y) * g.nx + x);
    }
    return acc;
}

// optical depth of a long ray (taps ordered along the ray, so consecutive
// offsets differ by at most one cell per axis): the column is wrapped once
// and then followed incrementally
template <typename T>
__device__ __forceinline__ T ray_sum(const GridC &g, const DTap *__restrict__ taps, const T *__restrict__ len,
                                     const T *__restrict__ mu_e, int off, int n, int bx, int by, int bz) {
    T acc = T(0);
    if (n == 0) return acc;
    DTap p = taps[off];
    int x = wrap_any(bx + p.dx, g.nx), y = wrap_any(by + p.dy, g.ny);
#pragma unroll 4
    for (int t = 0; t < n; ++t) {
        DTap tp = taps[off + t];
        x = wrap_small(x + (tp.dx - p.dx), g.nx);
        y = wrap_small(y + (tp.dy - p.dy), g.ny);
        p = tp;
        acc += len[off + t] * __ldg(mu_e + ((bz + tp.dz) * g.ny + y) * g.nx + x);
    }
    return acc;
}

// Optical depth of a long ray summed by a group of kRayLanes consecutive
// lanes: lane s of the group adds the taps t = s (mod kRayLanes), then the
// group combines its partial sums with a fixed butterfly (every lane gets
// the same bits).  Every lane of the warp must call it.
constexpr int kRayLanes = 4;
template <typename T>
__device__ __forceinline__ T ray_sum_lanes(const GridC &g, const RTap *__restrict__ taps, const T *__restrict__ len,
                                           const T *__restrict__ mu_e, int off, int n, int bx, int by) {
    const int s = threadIdx.x & (kRayLanes - 1);
    T acc = T(0);
#pragma unroll 2
    for (int t = s; t < n; t += kRayLanes) {
        const int2 r = __ldg(reinterpret_cast<const int2 *>(taps + off + t));
        int x = bx + (r.x & 0xffff);
        x -= x >= g.nx ? g.nx : 0;
        int y = by + (r.x >> 16);
        y -= y >= g.ny ? g.ny : 0;
        acc += __ldg(len + off + t) * __ldg(mu_e + r.y + y * g.nx + x);
    }
#pragma unroll
    for (int o = 1; o < kRayLanes; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

template <typename T>
__device__ __forceinline__ T hg(T g, T mu) {
    T d = T(1) + g * g - T(2) * g * mu;
    return (T(1) - g * g) / (T(4.0 * 3.14159265358979323846) * d * dsqrt<T>(d));
}

// segment table entry of canonical direction tab at node (x, y, z), x and y in range
template <typename T>
__device__ __forceinline__ T seg_at(const GridC &g, const T *__restrict__ tseg, int tab, int x, int y, int z) {
    return __ldg(tseg + (size_t)tab * g.npad + halo_pos(g, x, y, z));
}

template <typename T>
__device__ __forceinline__ T aslot_q(const ASlot &d) {
    if constexpr (sizeof(T) == 4) return d.q;
    else return d.qd;
}
template <typename T>
__device__ __forceinline__ T aslot_dinv(const ASlot &d) {
    if constexpr (sizeof(T) == 4) return d.dinv;
    else return d.dinvd;
}
template <typename T>
__device__ __forceinline__ T aslot_split(const ASlot &d) {
    if constexpr (sizeof(T) == 4) return d.split;
    else return d.splitd;
}

// The slot template of a layer staged in shared memory by the edge kernels:
// per slot its descriptor words (FP32: the first 64 bytes of ASlot; FP64:
// all 96) and 2 S constants, q^sun per species (a ground source: q in the
// first) and the HG weight toward the instrument per species (0 on the
// ground row).  Every thread of the block takes part; the caller
// synchronises the block before reading.
template <typename T>
__host__ __device__ constexpr int aslot_words() { return sizeof(T) == 4 ? 4 : 6; }
template <typename T>
inline size_t template_smem(const GridC &g) {
    return (size_t)g.ntmax * (16 * aslot_words<T>() + 2 * g.S * sizeof(T));
}
template <typename T, int S>
__device__ __forceinline__ void stage_template(const GridC &g, const GraphP &gp, const FieldP<T> &f, int t0, int nt,
                                               bool ground_row, int4 *sdesc, T *sconst) {
    constexpr int NW = aslot_words<T>();
    const int ndir = g.nd + g.ngd;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const int4 *src = reinterpret_cast<const int4 *>(gp.aslot + t0 + t);
        int4 d[NW];
#pragma unroll
        for (int e = 0; e < NW; ++e) d[e] = __ldg(src + e);
#pragma unroll
        for (int e = 0; e < NW; ++e) sdesc[(size_t)t * NW + e] = d[e];
        const int bits = d[1].z, dir = d[1].w, hgdir = d[2].x;
        const bool gsrc = (bits >> 11) & 1;
        T q;
        if constexpr (sizeof(T) == 4) q = __int_as_float(d[3].y);
        else q = __longlong_as_double(((long long)d[4].y << 32) | (unsigned)d[4].x);
#pragma unroll
        for (int sp = 0; sp < S; ++sp) {
            sconst[(size_t)t * 2 * S + sp] = !gsrc ? f.q_sun[sp * g.nd + dir] : (sp == 0 ? q : T(0));
            sconst[(size_t)t * 2 * S + S + sp] = ground_row ? T(0) : f.hgv[sp * ndir + hgdir];
        }
    }
}
// descriptor fields of staged slot t: a0, a1, a2 and (hit_off, q, dinv, split)
template <typename T>
struct StagedSlot {
    int4 a0, a1, a2;
    int hit_off;
    T q, dinv, split;
};
template <typename T>
__device__ __forceinline__ StagedSlot<T> staged_slot(const int4 *sdesc, int t) {
    constexpr int NW = aslot_words<T>();
    const int4 *d = sdesc + (size_t)t * NW;
    StagedSlot<T> o;
    o.a0 = d[0];
    o.a1 = d[1];
    o.a2 = d[2];
    if constexpr (sizeof(T) == 4) {
        const float4 a3 = reinterpret_cast<const float4 *>(d)[3];
        o.hit_off = __float_as_int(a3.x);
        o.q = a3.y;
        o.dinv = a3.z;
        o.split = a3.w;
    } else {
        o.hit_off = d[3].x;
        const double2 b0 = reinterpret_cast<const double2 *>(d)[4];
        const double2 b1 = reinterpret_cast<const double2 *>(d)[5];
        o.q = b0.x;
        o.dinv = b0.y;
        o.split = b1.x;
    }
    return o;
}

// optical depth of a tap list based at haloed position b
template <typename T>
__device__ __forceinline__ T tap_sum_h(const GraphP &gp, const T *__restrict__ mu_e_h, int off, int n, int b) {
    const T *len = tap_len<T>(gp);
    T acc = T(0);
    for (int t = 0; t < n; ++t) acc += len[off + t] * __ldg(mu_e_h + b + __ldg(gp.tap_h + off + t));
    return acc;
}

}  // namespace tk
