// Anisotropic multiple scattering (the edge unknowns of Eq. flux_system; see
// aniso.h for the recurrence and its factored form).  Layouts: X and Xn are
// [nin][n_nodes] (plane per arrival direction, rows = node ids), the
// per-node tables are transposed ([direction][node]) so that a warp's 32
// nodes read and write 128 contiguous bytes, L is haloed [nd][npad] so the
// transport pass reads it at the source-relative positions of the slot
// descriptors, and val holds the raw deposit fractions P in K's slot-major
// layout.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "aniso.h"
#include "aniso_contract.cuh"
#include "asm_util.cuh"
#include "kern.h"
#include "stage.cuh"

namespace tk {

// ---- double-single (FP32 pair) arithmetic of the refinement: a value is
// hi + lo with |lo| below half an ulp of hi; every step rounds to nearest
// (no contraction), the products exact by FMA ----
__device__ __forceinline__ float2 ds_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return make_float2(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ float2 ds_fast_norm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 ds_add(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x), bb = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    return ds_fast_norm(s, e);
}
__device__ __forceinline__ float2 ds_mul_f(float2 a, float b) {
    const float p = __fmul_rn(a.x, b);
    const float e = __fmaf_rn(a.y, b, __fmaf_rn(a.x, b, -p));
    return ds_fast_norm(p, e);
}
__device__ __forceinline__ float2 ds_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
    return ds_fast_norm(p, e);
}

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
// ground weights (the G of the folded form; their Cf is 1), plus Lsun where
// `sun` is set.  Block = 32 ground nodes x 8 warps: the warps sum
// interleaved arrival directions, then write interleaved ground directions
// (a warp's 32 nodes are adjacent).
template <typename T, typename XT, typename LT>
__global__ void __launch_bounds__(256) k_ani_ground(GridC g, AniP<T> a, const XT *__restrict__ X, LT *Lh, int sun,
                                                    const int *ctl) {
    __shared__ XT part[8][33];
    if (ctl && *(volatile const int *)ctl) return;
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool ok = c < g.n_ground;
    const int j = g.n_atm + c;
    const int nin = g.nd + g.ngd;
    XT s = XT(0);
    if (ok)
        for (int w = wv; w < nin; w += 8) s += X[(size_t)w * a.ldx + j];
    part[wv][lane] = s;
    __syncthreads();
    if (!ok) return;
    XT xt = XT(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) xt += part[i][lane];
    const int y = c / g.nx, x = c - y * g.nx;
    for (int k = wv; k < g.ngd; k += 8) {
        LT l = (LT)xt * (LT)a.Wg[(size_t)c * g.ngd + k];
        if (sun) l += (LT)a.LsT[(size_t)k * g.n_nodes + j];
        store_halo(Lh + (size_t)k * g.npad, g, x, y, g.nz, l);
    }
}

// The series' ground leave: G(k, c) = x_t(c) q_lamb_k c_k from the totals the
// last transport left in a.xtg (one thread per ground node and direction)
template <typename T>
__global__ void k_ani_ground_x(GridC g, AniP<T> a, T *Lh, const int *ctl) {
    if (ctl && *(volatile const int *)ctl) return;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.n_ground * g.ngd) return;
    const int k = idx / g.n_ground, c = idx - k * g.n_ground;
    const int y = c / g.nx, x = c - y * g.nx;
    store_halo(Lh + (size_t)k * g.npad, g, x, y, g.nz, a.xtg[c] * a.Wg[(size_t)c * g.ngd + k]);
}

// The same for the refinement's residual, in double-single: L = Lsun +
// (sum_w X) q_lamb c with X and L FP32 pairs.
__global__ void __launch_bounds__(256) k_ani_ground_ds(GridC g, AniP<float> a, const float2 *__restrict__ X,
                                                       float2 *Lh) {
    __shared__ float2 part[8][33];
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    const bool ok = c < g.n_ground;
    const int j = g.n_atm + c;
    const int nin = g.nd + g.ngd;
    float2 s = make_float2(0.f, 0.f);
    if (ok)
        for (int w = wv; w < nin; w += 8) s = ds_add(s, X[(size_t)w * a.ldx + j]);
    part[wv][lane] = s;
    __syncthreads();
    if (!ok) return;
    float2 xt = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 8; ++i) xt = ds_add(xt, part[i][lane]);
    const int y = c / g.nx, x = c - y * g.nx;
    for (int k = wv; k < g.ngd; k += 8) {
        const float2 l = ds_add(ds_mul_f(xt, a.Wg[(size_t)c * g.ngd + k]),
                                make_float2(a.LsT[(size_t)k * g.n_nodes + j], 0.f));
        store_halo(Lh + (size_t)k * g.npad, g, x, y, g.nz, l);
    }
}

// Transport as a gather: block = one group of 128 receiver rows (the edge
// kernel's lane quads), warp w sums the arrival directions w, w + kAniW, ...
// over the template's slots of that direction (tperm / tseg order), so
// every X(i, w) is written once, in a fixed order.
//   MODE 0: Xn = [radd] + rho sum P L, and the change against Xold
//   MODE 1: Xn = rho sum P L - X with L and X double-single pairs (float2),
//           the sums in double-single, the residual stored rounded to FP32
// Per-block sums of the squared change (residual) and of the squares of Xn
// (X64) go to a.part.
// The layer's slot order and direction runs are staged in shared memory
// first (dynamic: a.max_nt int4 then nin + 1 ints).
constexpr int kAniW = 8;
//   Pv: the deposit fractions (P' of the folded form, or P); bsrc, radd:
//   added to Xn where not null; Xold null: no change sums (d2 = 0)
template <typename T, int MODE, typename LT, typename XT>
__global__ void __launch_bounds__(32 * kAniW) k_ani_transport(GridC g, GraphP gp, FieldP<T> f, ViewC vc, AniP<T> a,
                                                              const T *__restrict__ Pv, const LT *__restrict__ Lh,
                                                              const XT *__restrict__ Xold, T *__restrict__ Xn,
                                                              const T *__restrict__ radd,
                                                              const T *__restrict__ bsrc, int check, double tol,
                                                              int term) {
    __shared__ double red[2][kAniW];
    extern __shared__ int4 tsm[];
    if (MODE == 0 && *(volatile const int *)a.ctl) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nin = g.nd + g.ngd;
    const GroupRows G = group_rows(g, gp, blockIdx.x);
    int4 *slots = tsm;
    int *seg = (int *)(tsm + a.max_nt);
    for (int i = threadIdx.x; i < G.nt; i += blockDim.x) slots[i] = __ldg(a.tslot + G.t0 + i);
    for (int i = threadIdx.x; i <= nin; i += blockDim.x) seg[i] = __ldg(a.tseg + (size_t)G.z * (nin + 1) + i);
    __syncthreads();
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
    // the change sums: per thread in the accumulation type of the term (the
    // stopping test needs no more; FP64 arithmetic is slow on this part)
    using D = T;
    D d2 = D(0), n2 = D(0);
    T gsum[4] = {T(0), T(0), T(0), T(0)};  // ground rows: sum over this warp's directions
    for (int d = w; d < nin; d += kAniW) {
        const int e0 = seg[d], e1 = seg[d + 1];
        // this direction's other operands first, so that their loads overlap the gathers
        XT xo[4];
        T add[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const size_t q = (size_t)d * a.ldx + (G.row[k] >= 0 ? G.row[k] : 0);
            xo[k] = Xold ? Xold[q] : XT{};
            add[k] = (MODE == 0 ? (radd ? radd[q] : T(0)) + (bsrc ? bsrc[q] : T(0)) : T(0));
        }
        LT acc[4];
        float acl[4] = {0.f, 0.f, 0.f, 0.f};  // MODE 1: the low words (acc holds the high ones)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = LT{};
        for (int e = e0; e < e1; ++e) {
            const int4 sl = slots[e];  // {t, src, dir, 0}
            T P[4];
            ld_quad(vrow + (size_t)sl.x * kGroup, P);
            const LT *Ld = Lh + (size_t)sl.z * g.npad + sl.y;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (G.row[k] < 0) continue;
                if constexpr (MODE == 1) {
                    const float2 l = __ldg(Ld + G.rp[k]);
                    ds_fma(acc[k].x, acl[k], l.x, l.y, P[k]);
                } else {
                    acc[k] += (LT)P[k] * __ldg(Ld + G.rp[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (G.row[k] < 0) continue;
            const size_t q = (size_t)d * a.ldx + G.row[k];
            if constexpr (MODE == 0) {
                const T xn = rho[k] * (T)acc[k] + add[k];
                const T dx = Xold ? xn - (T)xo[k] : T(0);
                gsum[k] += xn;
                Xn[q] = xn;
                d2 += dx * dx;
                n2 += xn * xn;
            } else {  // r = rho (acc + acl) - x in double-single, stored rounded to FP32
                const float2 t = ds_mul_f(ds_fast_norm(acc[k].x, acl[k]), rho[k]);
                const float2 r = ds_add(t, make_float2(-xo[k].x, -xo[k].y));
                const float rf = __fadd_rn(r.x, r.y);
                gsum[k] += rf;
                Xn[q] = rf;
                d2 += rf * rf;
                n2 += xo[k].x * xo[k].x;
            }
        }
    }
    // ground rows: the sum of the new X over the arrival directions (the next
    // term's ground leave), reduced over the warps in a fixed order
    if (ground_row && a.xtg != nullptr) {
        __shared__ T xs[kAniW][kGroup];
#pragma unroll
        for (int k = 0; k < 4; ++k) xs[w][lane + 32 * k] = gsum[k];
        __syncthreads();
        const int r = ((int)blockIdx.x - G.z * g.gpl) * kGroup + (int)threadIdx.x;  // row within the layer
        if (threadIdx.x < kGroup && r < g.nxy) {
            T t = T(0);
#pragma unroll
            for (int i = 0; i < kAniW; ++i) t += xs[i][threadIdx.x];
            a.xtg[r] = t;
        }
    }
    double d2d = (double)d2, n2d = (double)n2;
    for (int o = 16; o > 0; o >>= 1) {
        d2d += __shfl_xor_sync(0xffffffffu, d2d, o);
        n2d += __shfl_xor_sync(0xffffffffu, n2d, o);
    }
    if (lane == 0) {
        red[0][w] = d2d;
        red[1][w] = n2d;
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
    if (!check) return;
    // the last block to finish sums the partials in a fixed order (so the
    // result does not depend on which block that is) and takes the stopping
    // test (check 1: the series' a.ctl = {1, term} at the first change <= tol)
    __shared__ int last;
    __shared__ double s0[32 * kAniW], s1[32 * kAniW];
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(a.ctl + 2, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    double p0 = 0.0, p1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        p0 += __ldcg(a.part + 2 * (size_t)i);
        p1 += __ldcg(a.part + 2 * (size_t)i + 1);
    }
    s0[threadIdx.x] = p0;
    s1[threadIdx.x] = p1;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            s0[threadIdx.x] += s0[threadIdx.x + h];
            s1[threadIdx.x] += s1[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double rel = s1[0] > 0.0 ? sqrt(s0[0] / s1[0]) : 0.0;
        a.acc[0] = s0[0];
        a.acc[1] = s1[0];
        a.acc[2] = rel;
        if (check == 1 && rel <= tol) {
            a.ctl[0] = 1;
            a.ctl[1] = term;
        }
        a.ctl[2] = 0;  // the next launch counts again
    }
}

// Haloed planes of the routing coupling Cf (C where the routing applies and
// the chain has a receiver, else 1; ground sources 1) and of Lsun.
template <typename T>
__global__ void k_ani_planes(GridC g, GraphP gp, AniP<T> a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_nodes) return;
    const int z = j / g.nxy, r = j - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    if (j < g.n_atm) {
        const bool routed = a.on[j] > T(0);
        for (int u = 0; u < g.nd; ++u) {
            const bool has = z + gp.dirs[u].z < g.nz;
            const T cf = (routed && has) ? a.CT[(size_t)u * g.n_atm + j] : T(1);
            store_halo(a.CfH + (size_t)u * g.npad, g, x, y, z, cf);
            store_halo(a.Lh + (size_t)u * g.npad, g, x, y, z, a.LsT[(size_t)u * g.n_nodes + j]);
        }
    } else {
        for (int k = 0; k < g.ngd; ++k) {
            store_halo(a.CfH + (size_t)k * g.npad, g, x, y, z, T(1));
            store_halo(a.Lh + (size_t)k * g.npad, g, x, y, z, a.LsT[(size_t)k * g.n_nodes + j]);
        }
    }
}

// P' = P Cf(src, dir) for every slot, in K's value layout (block = one
// group of 128 rows, as the transport walks them)
template <typename T>
__global__ void __launch_bounds__(128) k_ani_pc(GridC g, GraphP gp, FieldP<T> f, AniP<T> a) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const GroupRows G = group_rows(g, gp, blockIdx.x);
    for (int t = w; t < G.nt; t += 4) {
        const ASlot &sd = gp.aslot[G.t0 + t];
        const int src = __ldg(&sd.src), dir = __ldg(&sd.dir);
        const size_t v0 = (size_t)G.vb + (size_t)t * kGroup + 4 * lane;
        const T *cf = a.CfH + (size_t)dir * g.npad + src;
#pragma unroll
        for (int k = 0; k < 4; ++k) a.Pc[v0 + k] = G.row[k] >= 0 ? f.val[v0 + k] * __ldg(cf + G.rp[k]) : T(0);
    }
}

__global__ void k_ani_update(long long n, const float *e, float2 *X, int init) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        X[i] = init ? make_float2(e[i], 0.f) : ds_add(X[i], make_float2(e[i], 0.f));
}

__device__ __forceinline__ double as_double(float v) { return (double)v; }
__device__ __forceinline__ double as_double(double v) { return v; }
__device__ __forceinline__ double as_double(float2 v) { return (double)v.x + (double)v.y; }

// x = sum_w X(i, w) into the FP64 haloed vector, and the emission toward the
// instrument E_i = e1_i Theta_i(s0 . v) + sum_w Theta_i(w . v) X(i, w)
template <typename T, typename XT>
__global__ void k_aniso_finish(GridC g, FieldP<T> f, const XT *__restrict__ X, int ldx, double *x64, T *emis) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_nodes) return;
    const int nin = g.nd + g.ngd;
    const int z = i / g.nxy, r = i - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    if constexpr (std::is_same<XT, float2>::value) {
        // FP32 pairs: the sums in pairs as well (FP64 arithmetic is slow on this part)
        float2 xt = make_float2(0.f, 0.f);
        for (int wv = 0; wv < nin; ++wv) xt = ds_add(xt, X[(size_t)wv * ldx + i]);
        store_halo(x64, g, x, y, z, (double)xt.x + (double)xt.y);
        if (i >= g.n_atm) return;
        float w[MAX_SPECIES];
        float th0 = 0.f;
        for (int sp = 0; sp < g.S; ++sp) {
            w[sp] = f.wsp[(size_t)sp * g.n_atm + i];
            th0 += w[sp] * f.hg0v[sp];
        }
        float eh = 0.f, el = 0.f;
        for (int wv = 0; wv < nin; ++wv) {
            const float2 xw = X[(size_t)wv * ldx + i];
            float th = 0.f;
            for (int sp = 0; sp < g.S; ++sp) th += w[sp] * f.hgv[sp * nin + wv];
            ds_fma(eh, el, xw.x, xw.y, th);
        }
        emis[i] = (T)((double)f.e1[i] * (double)th0 + (double)eh + (double)el);
    } else {
        double xt = 0.0;
        for (int wv = 0; wv < nin; ++wv) xt += as_double(X[(size_t)wv * ldx + i]);
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
            const double xw = as_double(X[(size_t)wv * ldx + i]);
            if (xw == 0.0) continue;
            double th = 0;
            for (int sp = 0; sp < g.S; ++sp) th += w[sp] * (double)f.hgv[sp * nin + wv];
            e += th * xw;
        }
        emis[i] = (T)((double)f.e1[i] * th0 + e);
    }
}

// ---- launchers ----
namespace {

// cuTensorMapEncodeTiled, from the driver through the runtime (no link to
// the driver library)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// a [rows][ld] FP32 array as a 2-D tensor map of n_inner x rows, boxes of
// 128 x kAniRows, zero beyond the array
bool rows_map(CUtensorMap &m, const float *base, int n_inner, int ld, int rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || (ld % 4) || ((uintptr_t)base % 16)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)n_inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kAniTileM, (cuuint32_t)kAniRows};
    const cuuint32_t es[2] = {1, 1};
    return enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tensor-core launch of the leave contraction: N padded to one of a few
// tile widths (N <= 128), S <= MAX_SPECIES.  cudaErrorInvalidValue when the
// tensor maps of X and zf cannot be made.
template <class Op>
cudaError_t mma_leave(cudaStream_t st, const Op &op, int S, int R, int N, const float *B, const int *ctl,
                      int *status) {
    CUtensorMap mx, mz;
    if (!rows_map(mx, op.X, op.g.n_atm, op.ldx, R) || !rows_map(mz, op.zf, op.g.n_atm, op.ldz, R))
        return cudaErrorInvalidValue;
    const int np = ani_leave_np(N, S);
#define TK_L(SS, NN) ani_mma_launch<SS, NN, Op>(st, op, R, N, B, mx, mz, ctl, status)
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
    return cudaSuccess;
}

// first node of the layers from which some direction has no receiver
// (the top max(uz) layers)
inline int top_begin(const GridC &g) { return std::max(0, g.nz - g.R) * g.nxy; }

template <typename T>
size_t transport_smem(const GridC &g, const AniP<T> &a) {
    return (size_t)a.max_nt * sizeof(int4) + (size_t)(g.nd + g.ngd + 1) * sizeof(int);
}

// the leave contraction; with_top adds the top layers' tiles
template <typename T>
LeaveOp<T, T, T, true> leave_op(const GridC &g, const GraphP &gp, const AniP<T> &a, const T *wsp, const T *X, int sun,
                                bool with_top) {
    LeaveOp<T, T, T, true> op;
    op.g = g;
    op.jtop = with_top ? top_begin(g) / kAniTileM * kAniTileM : g.n_atm;  // tiles start on 128 nodes
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
    op.ldx = a.ldx;
    op.ldz = a.ldz;
    return op;
}
template <typename T>
SqcOp<T> sqc_op(const GridC &g, const AniP<T> &a, const T *wsp) {
    SqcOp<T> op;
    op.g = g;
    op.jtop = g.n_atm;
    op.CT = a.CT;
    op.wsp = wsp;
    op.on = a.on;
    op.SQ = a.SQ;
    op.Q = a.Q;
    op.zf = a.zf;
    op.ldz = a.ldz;
    return op;
}

// the contractions with their raw outputs out[n][n_atm] (tests)
template <class Base>
struct RawOp : Base {
    static constexpr bool kBatched = false;
    float *raw;
    struct Pre {};
    __device__ __forceinline__ Pre pre(int) const { return Pre{}; }
    template <typename V>
    __device__ __forceinline__ void out(const Pre &, int j, int n, V val, bool) const {
        raw[(size_t)n * this->g.n_atm + j] = (float)val;
    }
};

}  // namespace

template <typename T>
void launch_aniso_prep(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const ViewP &vp, const AniP<T> &a, bool tables, long long *launches) {
    const int nin = g.nd + g.ngd;
    const long long warps = (long long)g.S * nin * g.nd;
    if (tables) {
        k_aniso_qcells<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(g, vc, vp, a.Qraw);
        k_aniso_qnorm<T><<<(g.S * nin + 127) / 128, 128, 0, st>>>(g, a.Qraw, a.Q);
        k_ani_sq<T><<<(g.nz * g.S * nin + 127) / 128, 128, 0, st>>>(g, gp, a.Q, a.SQ);
        if (launches) *launches += 3;
    }
    k_aniso_couple<T><<<(g.n_nodes + 127) / 128, 128, 0, st>>>(g, gp, f, vc, a);
    // the routing denominators on the CUDA cores: zf is part of the operator
    // the FP64 residual refines against, so it keeps FP32 sums
    ani_simt_launch<T>(st, sqc_op<T>(g, a, f.wsp), g.S, g.nd, nin, nullptr);
    // the folded form: Cf and Lsun planes, P' = P Cf, b = rho T Lsun
    const int nblk = (g.nz + 1) * g.gpl;
    cudaMemsetAsync(a.ctl, 0, 3 * sizeof(int), st);  // the transport below must not see a converged flag
    k_ani_planes<T><<<(g.n_nodes + 127) / 128, 128, 0, st>>>(g, gp, a);
    k_ani_pc<T><<<nblk, 128, 0, st>>>(g, gp, f, a);
    AniP<T> ab = a;  // the ground sums of b go to xtb
    ab.xtg = a.xtb;
    k_ani_transport<T, 0, T, T><<<nblk, 32 * kAniW, transport_smem(g, a), st>>>(g, gp, f, vc, ab, f.val, a.Lh, nullptr,
                                                                                  a.b, nullptr, nullptr, 0, 0.0, 0);
    if (launches) *launches += 5;
    if constexpr (sizeof(T) == 4) {
        if (tables && a.mma) {
            const LeaveOp<T, T, T, true> lop = leave_op<T>(g, gp, a, f.wsp, nullptr, 0, false);
            const int np = ani_leave_np(g.nd, g.S);
            using LO = LeaveOp<T, T, T, true>;
            if (g.S == 1) k_ani_pack<LO, 8><<<256, 256, 0, st>>>(lop, nin, g.nd, np, a.Bl);
            else if (g.S == 2) k_ani_pack<LO, 16><<<256, 256, 0, st>>>(lop, nin, g.nd, np, a.Bl);
            else if (g.S == 3) k_ani_pack<LO, 24><<<256, 256, 0, st>>>(lop, nin, g.nd, np, a.Bl);
            else k_ani_pack<LO, 32><<<256, 256, 0, st>>>(lop, nin, g.nd, np, a.Bl);
            if (launches) *launches += 1;
        }
    }
}

template <typename T>
cudaError_t launch_aniso_leave(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f,
                               const AniP<T> &a, const T *X, long long *launches) {
    const int nin = g.nd + g.ngd;
    const LeaveOp<T, T, T, true> lop = leave_op<T>(g, gp, a, f.wsp, X, 0, true);
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        if (a.mma) {
            const cudaError_t e = mma_leave(st, lop, g.S, nin, g.nd, a.Bl, a.ctl, f.status);
            if (e != cudaSuccess) return e;
            done = true;
        }
    }
    if (!done) ani_simt_launch<T>(st, lop, g.S, nin, g.nd, a.ctl);
    if (g.n_ground > 0)
        k_ani_ground_x<T><<<(g.n_ground * g.ngd + 255) / 256, 256, 0, st>>>(g, a, a.Lh, a.ctl);
    if (launches) *launches += g.n_ground > 0 ? 2 : 1;
    return cudaSuccess;
}

template <typename T>
void launch_aniso_move(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const AniP<T> &a, const T *X, T *Xn, const T *radd, bool sun, double tol, int term,
                       long long *launches) {
    const int nblk = (g.nz + 1) * g.gpl;
    k_ani_transport<T, 0, T, T><<<nblk, 32 * kAniW, transport_smem(g, a), st>>>(g, gp, f, vc, a, a.Pc, a.Lh, X, Xn, radd,
                                                                                  sun ? a.b : nullptr, 1, tol, term);
    if (launches) *launches += 1;
}

// ---- the residual's contraction in double-single ----
// A = w_sp zf X (top layers: w_sp X) in double-single from the pairs of X,
// once per residual, into [Kp][ld] (k = w S + sp, zero past the nodes and
// past K), so that the contraction stages its operands with plain
// asynchronous copies.
constexpr int kDsM = 64, kDsN = 128, kDsK = 16;  // tile nodes, columns, K chunk
__global__ void k_ani_asplit(GridC g, const float *__restrict__ wsp, const float *__restrict__ zf, int ldz,
                             const float2 *__restrict__ X, int ldx, int S, int Kp, int j0, int nj, int ld,
                             int with_zf, float2 *A) {
    const int nin = g.nd + g.ngd;
    const long long total = (long long)Kp * ld;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(idx / ld), jj = (int)(idx - (long long)k * ld);
        const int r = k / S, sp = k - r * S, j = j0 + jj;
        float2 v = make_float2(0.f, 0.f);
        if (r < nin && jj < nj) {
            const float w = wsp[(size_t)sp * g.n_atm + j];
            const float2 wz = with_zf ? ds_two_prod(w, zf[(size_t)r * ldz + j]) : make_float2(w, 0.f);
            v = ds_mul(wz, X[(size_t)r * ldx + j]);
        }
        A[idx] = v;
    }
}
// B((w, sp), u) = Q_sp(w -> u) in [Kp][kDsN] (zero past nd and K)
__global__ void k_ani_bpad(const float *__restrict__ Q, int S, int nin, int nd, int Kp, float *B) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Kp * kDsN) return;
    const int k = idx / kDsN, n = idx - k * kDsN, r = k / S, sp = k - r * S;
    B[idx] = (r < nin && n < nd) ? Q[((size_t)sp * nin + r) * nd + n] : 0.f;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Tile of 64 nodes x 128 columns, 512 threads, thread (tx, ty) = (tid % 16,
// tid / 16) accumulating nodes 4 tx .. + 3 times columns 4 ty .. + 3 in
// double-single (many warps per SM: the two-sum chains are serial); K in
// chunks of 16 staged by cp.async, two stages.  The first ntop tiles are the
// top layers' (A from At, nodes from jtop).
constexpr int kDsThreads = 512;
__global__ void __launch_bounds__(kDsThreads, 1) k_ani_ds(GridC g, AniP<float> ap, const int4 *__restrict__ dirs,
                                                          int jtop, const float2 *__restrict__ Am, int ldm,
                                                          const float2 *__restrict__ At, int ldt, int ntop,
                                                          const float *__restrict__ Bp, int Kp, int N, float2 *L) {
    __shared__ __align__(16) float2 As[2][kDsK][kDsM];
    __shared__ __align__(16) float Bs[2][kDsK][kDsN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const bool top = (int)blockIdx.x < ntop;
    const int t0 = top ? (int)blockIdx.x * kDsM : ((int)blockIdx.x - ntop) * kDsM;  // column in A
    const int j0 = (top ? jtop : 0) + t0;
    const float2 *A = top ? At : Am;
    const int lda = top ? ldt : ldm;
    auto stage = [&](int c, int b) {
        const int row = tid >> 5, c16 = tid & 31;  // 512 copies of 16 bytes for each operand
        cp_async16(&As[b][row][2 * c16], A + (size_t)(c * kDsK + row) * lda + t0 + 2 * c16);
        cp_async16(&Bs[b][row][4 * c16], Bp + (size_t)(c * kDsK + row) * kDsN + 4 * c16);
        cp_async_commit();
    };
    float acc[4][4], acl[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = acl[p][q] = 0.f;
    const int nch = Kp / kDsK;
    stage(0, 0);
    for (int c = 0; c < nch; ++c) {
        if (c + 1 < nch) {
            stage(c + 1, (c + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int b = c & 1;
        if (4 * ty < N) {  // column groups entirely past N have nothing to add
#pragma unroll 4
            for (int k = 0; k < kDsK; ++k) {
                const float4 a01 = *reinterpret_cast<const float4 *>(&As[b][k][4 * tx]);
                const float4 a23 = *reinterpret_cast<const float4 *>(&As[b][k][4 * tx + 2]);
                const float4 bq = *reinterpret_cast<const float4 *>(&Bs[b][k][4 * ty]);
                const float ah[4] = {a01.x, a01.z, a23.x, a23.z}, al[4] = {a01.y, a01.w, a23.y, a23.w};
                const float bv[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) ds_fma(acc[p][q], acl[p][q], ah[p], al[p], bv[q]);
            }
        }
        __syncthreads();  // the stage is read before it is refilled
    }
    // L = Lsun + Cf G in double-single: main tiles the directions with a
    // receiver (Cf = C where the routing applies), top tiles the others (Cf = 1)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int j = j0 + 4 * tx + p;
        if (j >= g.n_atm) continue;
        const int z = j / g.nxy, rr = j - z * g.nxy, y = rr / g.nx, x = rr - y * g.nx;
        const bool routed = ap.on[j] > 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int n = 4 * ty + q;
            if (n >= N) continue;
            const bool has = z + __ldg(&dirs[n].z) < g.nz;
            if (top == has) continue;
            const float cf = (routed && has) ? ap.CT[(size_t)n * g.n_atm + j] : 1.f;
            const float2 v = ds_fast_norm(acc[p][q], acl[p][q]);
            const float2 l = ds_add(ds_mul_f(v, cf), make_float2(ap.LsT[(size_t)n * g.n_nodes + j], 0.f));
            store_halo(L + (size_t)n * g.npad, g, x, y, z, l);
        }
    }
}

void launch_aniso_resid(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<float> &f,
                        const ViewC &vc, const AniP<float> &a, const float2 *X, float2 *L, float *r,
                        long long *launches) {
    const int nin = g.nd + g.ngd;
    const int jtop = top_begin(g) / kAniTileM * kAniTileM;
    // A split in FP32 pairs (main and top layers), B padded, then the contraction
    const int Kp = ani_ds_kp(nin, g.S);
    const int ntop_nodes = g.n_atm - jtop, ldt = ani_ds_ldt(g, jtop);
    k_ani_asplit<<<2048, 256, 0, st>>>(g, f.wsp, a.zf, a.ldz, X, a.ldx, g.S, Kp, 0, g.n_atm, a.ldz, 1, a.Ads);
    k_ani_asplit<<<512, 256, 0, st>>>(g, f.wsp, a.zf, a.ldz, X, a.ldx, g.S, Kp, jtop, ntop_nodes, ldt, 0, a.Atop);
    k_ani_bpad<<<(Kp * kDsN + 255) / 256, 256, 0, st>>>(a.Q, g.S, nin, g.nd, Kp, a.Bds);
    const int ntop = (ntop_nodes + kDsM - 1) / kDsM;
    k_ani_ds<<<ntop + (g.n_atm + kDsM - 1) / kDsM, kDsThreads, 0, st>>>(g, a, gp.dirs, jtop, a.Ads, a.ldz, a.Atop,
                                                                        ldt, ntop, a.Bds, Kp, g.nd, L);
    if (g.n_ground > 0) k_ani_ground_ds<<<(g.n_ground + 31) / 32, 256, 0, st>>>(g, a, X, L);
    const int nblk = (g.nz + 1) * g.gpl;
    k_ani_transport<float, 1, float2, float2><<<nblk, 32 * kAniW, transport_smem(g, a), st>>>(
        g, gp, f, vc, a, f.val, L, X, r, nullptr, nullptr, 2, 0.0, 0);
    if (launches) *launches += g.n_ground > 0 ? 6 : 5;
}

void launch_aniso_update(cudaStream_t st, long long n, const float *e, float2 *X, bool init) {
    k_ani_update<<<1216, 256, 0, st>>>(n, e, X, init ? 1 : 0);
}

template <typename T, typename XT>
void launch_aniso_finish(cudaStream_t st, const GridC &g, const FieldP<T> &f, const XT *X, int ldx, double *x64,
                         T *emis, long long *launches) {
    k_aniso_finish<T, XT><<<(g.n_nodes + 127) / 128, 128, 0, st>>>(g, f, X, ldx, x64, emis);
    if (launches) *launches += 1;
}

template <typename XT>
__global__ void k_ani_export(GridC g, const XT *__restrict__ X, int ldx, double *out) {
    const long long n = (long long)(g.nd + g.ngd) * g.n_nodes;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(idx / g.n_nodes), j = (int)(idx - (long long)w * g.n_nodes);
        out[idx] = as_double(X[(size_t)w * ldx + j]);
    }
}
template <typename XT>
void launch_aniso_export(cudaStream_t st, const GridC &g, const XT *X, int ldx, double *out) {
    k_ani_export<XT><<<1216, 256, 0, st>>>(g, X, ldx, out);
}
template void launch_aniso_export<float2>(cudaStream_t, const GridC &, const float2 *, int, double *);
template void launch_aniso_export<double>(cudaStream_t, const GridC &, const double *, int, double *);

cudaError_t launch_aniso_contract_test(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<float> &f,
                                       const AniP<float> &a, const float *X, float *out, int which, bool mma) {
    const int nin = g.nd + g.ngd;
    if (which == 0) {
        RawOp<LeaveOp<float, float, float, true>> op;
        static_cast<LeaveOp<float, float, float, true> &>(op) = leave_op<float>(g, gp, a, f.wsp, X, 0, false);
        op.raw = out;
        if (mma) return mma_leave(st, op, g.S, nin, g.nd, a.Bl, nullptr, f.status);
        ani_simt_launch<float>(st, op, g.S, nin, g.nd, nullptr);
    } else {
        RawOp<SqcOp<float>> op;
        static_cast<SqcOp<float> &>(op) = sqc_op<float>(g, a, f.wsp);
        op.raw = out;
        ani_simt_launch<float>(st, op, g.S, g.nd, nin, nullptr);
    }
    return cudaSuccess;
}

#define INST(T)                                                                                                 \
    template void launch_aniso_prep<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,          \
                                       const ViewC &, const ViewP &, const AniP<T> &, bool, long long *);       \
    template cudaError_t launch_aniso_leave<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,  \
                                               const AniP<T> &, const T *, long long *);                        \
    template void launch_aniso_move<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,          \
                                       const ViewC &, const AniP<T> &, const T *, T *, const T *, bool, double, \
                                       int, long long *);                                                       \
    template void launch_aniso_finish<T, T>(cudaStream_t, const GridC &, const FieldP<T> &, const T *, int,     \
                                            double *, T *, long long *);
INST(float)
INST(double)
#undef INST
template void launch_aniso_finish<float, float2>(cudaStream_t, const GridC &, const FieldP<float> &,
                                                 const float2 *, int, double *, float *, long long *);

}  // namespace tk
