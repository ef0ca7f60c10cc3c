// Adjoint of the path: the gradient of J(L) with respect to the absorption
// coefficient mu_a of every voxel, given dJ/dL for every detector pixel.
//
// mu_a enters the path only through mu_e = mu_a + mu_s, and mu_e enters
//   - the optical depths of the chain segments, the tau_inf tables and the
//     direct beam (all linear in mu_e, through lattice taps and tap lists);
//   - the scattering ratio rho_i = mu_s / mu_e of every receiver row of K;
//   - e1_j = omega_j B T_sun,j (1 - exp(-mu_e hz / mu0)) with omega = mu_s / mu_e;
//   - the line-of-sight sums of the detector (attenuation and voxel weights).
// The adjoint runs the path backwards (reverse-mode differentiation of the
// forward kernels, written out by hand):
//   pixels  -> E-bar, x-bar (ground), e1-bar (ground), mu_e-bar (LOS terms)
//   E_i = e1_i theta0_i + g_i + sum_slots theta K x    -> x-bar += (theta K)^T E-bar
//   (I - K) x = s                                      -> (I - K)^T lambda = x-bar, s-bar = lambda
//   s_i, g_i and K_ij from P_ij, rho_i, e1_j           -> per slot P-bar, rho-bar, e1-bar
//   P from the optical depths                          -> tau-bar, scattered into the segment
//                                                         table, tau_inf, tap lists
//   tables and e1                                      -> mu_e-bar
// All sums over shared targets use atomic adds (the gradient is therefore
// reproducible to rounding, not bit for bit).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "asm_util.cuh"
#include "kern.h"
#include "select.h"
#include "stage.cuh"

namespace tk {

// sum of a haloed array over node (x, y, z)'s position and its halo copies
template <typename T>
__device__ __forceinline__ T gather_halo(const T *a, const GridC &g, int x, int y, int z) {
    const long long p = halo_pos(g, x, y, z);
    const int ax = x < g.H ? g.nx : (x >= g.nx - g.H ? -g.nx : 0);
    const int ay = y < g.H ? g.ny * g.nxp : (y >= g.ny - g.H ? -g.ny * g.nxp : 0);
    T v = a[p];
    if (ax) v += a[p + ax];
    if (ay) {
        v += a[p + ay];
        if (ax) v += a[p + ax + ay];
    }
    return v;
}

// mu_e-bar += w len over a tap list based at cell (bx, by, bz) (wrapped per tap)
template <typename T>
__device__ __forceinline__ void scatter_taps(const GridC &g, const DTap *__restrict__ taps, const T *__restrict__ len,
                                             int off, int n, int bx, int by, int bz, T w, T *mubar) {
    if (w == T(0)) return;
    for (int t = 0; t < n; ++t) {
        const DTap tp = taps[off + t];
        const int x = wrap_any(bx + tp.dx, g.nx), y = wrap_any(by + tp.dy, g.ny), z = bz + tp.dz;
        atomicAdd(mubar + (z * g.ny + y) * g.nx + x, w * len[off + t]);
    }
}

// same over a tap list addressed in the haloed layout from position b
template <typename T>
__device__ __forceinline__ void scatter_taps_h(const GraphP &gp, int off, int n, int b, T w, T *mubar_h) {
    if (w == T(0)) return;
    const T *len = tap_len<T>(gp);
    for (int t = 0; t < n; ++t) atomicAdd(mubar_h + b + __ldg(gp.tap_h + off + t), w * len[off + t]);
}

// ---------------------------------------------------------------------------
// K^T in the group-major layout of the transposed templates: entry e of
// source node j holds K_{i, t} with i = j - (sdx, sdy) (periodic) in the
// receiver layer of the entry.  One block per group of 128 source rows.

template <typename T>
__global__ void k_transpose_vals(GridC g, GraphP gp, TransP tp, const T *__restrict__ val, T *__restrict__ valT) {
    const int zs = blockIdx.x / g.gpl, q = blockIdx.x - zs * g.gpl;
    const int e0 = tp.tstart[zs], ne = tp.tstart[zs + 1] - e0;
    const long long vbT = tp.voff[zs] + (long long)q * ne * kGroup;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int e = w; e < ne; e += nw) {
        const int4 inf = __ldg(tp.info + e0 + e);  // (template-local index, receiver layer, sdx, sdy)
        const int zi = inf.y;
        const int nt = __ldg(gp.tstart + zi + 1) - __ldg(gp.tstart + zi);
        const long long vz = __ldg(gp.voff + zi);
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = q * kGroup + lane + 32 * k;
            v[k] = T(0);
            if (r < g.nxy) {
                const int y = r / g.nx, x = r - y * g.nx;
                const int ri = wrap_small(y - inf.w, g.ny) * g.nx + wrap_small(x - inf.z, g.nx);
                v[k] = val[val_base(vz, nt, ri) + (long long)inf.x * kGroup];
            }
        }
        st_quad(valT + vbT + (long long)e * kGroup + 4 * lane, v);
    }
}

// ---------------------------------------------------------------------------
// x-bar from the emission: x-bar_j += sum_{i, t: src = j} K_{i,t} theta_{i,t} E-bar_i
// over the transposed templates (rows = sources), with
// theta_{i,t} = sum_sp w_sp,i hg_sp(slot direction).
template <typename T, int S>
struct OpEmisT {
    using A = T;
    static constexpr int NA = 4;
    static constexpr bool kPart = false;
    struct Pre {
        T u;
    };
    struct Slot {
        T hv[S];
    };
    const T *Ebar_h, *wsp_h, *hgv;
    const int *hgdirT;
    T *xbar;
    long long npad;
    int ndir;
    __device__ __forceinline__ Slot slot(const GraphP &, int e) const {
        Slot si;
        const int h = __ldg(hgdirT + e);
#pragma unroll
        for (int sp = 0; sp < S; ++sp) si.hv[sp] = hgv[sp * ndir + h];
        return si;
    }
    __device__ __forceinline__ void add(A *a, int k, T v, int i, const Slot &si) const {
        T th = T(0);
#pragma unroll
        for (int sp = 0; sp < S; ++sp) th += __ldg(wsp_h + (size_t)sp * npad + i) * si.hv[sp];
        a[k] += v * __ldg(Ebar_h + i) * th;
    }
    __device__ __forceinline__ Pre pre(const GroupRows &G, int k) const {
        Pre p;
        p.u = xbar[G.row[k]];
        return p;
    }
    template <int W>
    __device__ __forceinline__ static void combine_row(const A (*sh)[NA][32], int lane, int k, A *a) {
        sum_word<W, A, NA>(sh, lane, k, a);
    }
    __device__ __forceinline__ double finish_row(const GroupRows &G, int k, const A *a, const Pre &p) const {
        xbar[G.row[k]] = p.u + a[k];
        return 0.0;
    }
};

// ---------------------------------------------------------------------------
// Pixels.  L_p = sum_m exp(-tau_m) F_m E_m / V + exp(-tau_tot) (e1_c + x_c) / (pi hx hy),
// F_m = (1 - exp(-mu_m ds_m)) / mu_m.  One warp per pixel, lanes over
// contiguous chunks of the line of sight as in the forward; a reverse walk of
// each chunk with the radiance beyond the current tap (suffix over later
// chunks plus the ground term) gives
//   dL/dE_m = exp(-tau_m) F_m / V
//   dL/dmu_m = exp(-tau_m) E_m F'_m / V - ds_m (radiance beyond tap m)
//   dL/de1_c = dL/dx_c = exp(-tau_tot) / (pi hx hy).
template <typename T>
__global__ void k_pix_adj(GridC g, FieldP<T> f, ViewC vc, ViewP vp, const T *__restrict__ emis,
                          const double *__restrict__ x, const T *__restrict__ Lbar, AdjP<T> ad) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (p >= vp.npx * vp.npy) return;
    const T lb = Lbar[p];
    const T *len;
    if constexpr (sizeof(T) == 4)
        len = (const T *)vp.los_len_f;
    else
        len = (const T *)vp.los_len_d;
    const int cx = vp.pix_cx[p], cy = vp.pix_cy[p], cl = vp.pix_cls[p];
    const int off = vp.los_off[cl], n = vp.los_n[cl];
    const T inv_vol = (T)(1.0 / (g.hx * g.hy * g.hz));
    const T inv_gnd = (T)(1.0 / (3.14159265358979323846 * g.hx * g.hy));
    const int per = (n + 31) / 32;
    const int t0 = min(n, lane * per), t1 = min(n, t0 + per);
    // pass 1: the chunk's optical depth and contribution as seen from its top
    T tau = T(0), L = T(0);
    for (int t = t0; t < t1; ++t) {
        const DTap tp = vp.los_taps[off + t];
        const int idx = (tp.dz * g.ny + wrap_any(cy + tp.dy, g.ny)) * g.nx + wrap_any(cx + tp.dx, g.nx);
        const T me = f.mu_e[idx], ds = len[off + t];
        const T fr = me > T(0) ? -dexpm1<T>(-me * ds) / me : ds;
        L += dexp<T>(-tau) * fr * emis[idx] * inv_vol;
        tau += me * ds;
    }
    T incl = tau;
    for (int o = 1; o < 32; o <<= 1) {
        const T v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const T before = incl - tau;
    const T total = __shfl_sync(0xffffffffu, incl, 31);
    const T A = dexp<T>(-before) * L;
    T suf = A;  // inclusive suffix over the lanes
    for (int o = 1; o < 32; o <<= 1) {
        const T v = __shfl_down_sync(0xffffffffu, suf, o);
        if (lane + o < 32) suf += v;
    }
    const int c = g.n_atm + cy * g.nx + cx;
    const T eg = dexp<T>(-total) * inv_gnd;
    const T G = eg * (f.e1[c] + (T)x[halo_pos(g, cx, cy, g.nz)]);
    // pass 2: reverse walk, S = radiance beyond the current tap
    T S = suf - A + G, rem = T(0);
    for (int t = t1 - 1; t >= t0; --t) {
        const DTap tp = vp.los_taps[off + t];
        const int idx = (tp.dz * g.ny + wrap_any(cy + tp.dy, g.ny)) * g.nx + wrap_any(cx + tp.dx, g.nx);
        const T me = f.mu_e[idx], ds = len[off + t];
        const T e = dexp<T>(-me * ds);
        const T fr = me > T(0) ? -dexpm1<T>(-me * ds) / me : ds;
        const T dfr = me > T(0) ? (ds * e - fr) / me : -T(0.5) * ds * ds;
        const T att = dexp<T>(-(before + (tau - rem - me * ds)));
        const T E = emis[idx];
        atomicAdd(ad.mubar + idx, lb * (att * E * inv_vol * dfr - ds * S));
        atomicAdd(ad.Ebar + idx, lb * att * fr * inv_vol);
        S += att * fr * E * inv_vol;
        rem += me * ds;
    }
    if (lane == 0) {
        atomicAdd(ad.e1bar + c, lb * eg);
        atomicAdd(ad.xbar + c, lb * eg);
    }
}

// ---------------------------------------------------------------------------
// Edge march backwards: per slot of every receiver row the deposit P and the
// weights are recomputed as in the forward edge kernel, and with
//   c = lambda_i + E-bar_i theta_{i,t}          (s-bar = lambda, g-bar = E-bar)
//   P-bar = rho_i c (x_j W^iso + W^sun e1_j)
// the adjoints go to rho_i, e1_j and the optical depths of the slot.
#ifndef TK_ADJ_W
#define TK_ADJ_W 4
#endif
// blocks per SM the register budget is sized for: 8 (64 registers) measured
// best on GB300 (gradient 1.380 -> 1.348 ms against the uncapped 96 registers)
#ifndef TK_ADJ_MINB
#define TK_ADJ_MINB 8
#endif
constexpr int kAdjW = TK_ADJ_W;  // warps per 128-row group of the reverse edge march
// kSel: coupling selection, the weights q c come from the planes wsi / wss
// (they depend on the scattering coefficients only, so absorption has no
// path through them)
template <typename T, int S, bool kSel>
__global__ void __launch_bounds__(32 * kAdjW, TK_ADJ_MINB)
    k_asm_adj(GridC g, GraphP gp, FieldP<T> f, ViewC vc, const double *__restrict__ x64,
              const double *__restrict__ lam64, AdjP<T> ad, const T *__restrict__ wsi, const T *__restrict__ wss) {
    constexpr int W = kAdjW;
    __shared__ T sh[W][4][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const GroupRows G = group_rows(g, gp, blockIdx.x);
    const bool ground_row = G.z == g.nz;
    const T rt_lamb = dsqrt<T>((T)(vc.albedo * __longlong_as_double((long long)*f.mus_max_bits)));
    const int ndir = g.nd + g.ngd;
    T rho[4], wr[4][S], lam[4], Eb[4], rhob[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int rc = G.row[k] >= 0 ? G.row[k] : G.z * g.nxy;
        rhob[k] = T(0);
        lam[k] = G.row[k] >= 0 ? (T)lam64[G.rp[k]] : T(0);
        if (!ground_row) {
            const T me = f.mu_e[rc], ms = f.mu_st[rc];
            rho[k] = me > T(0) ? ms / me : T(0);
            Eb[k] = G.row[k] >= 0 ? ad.Ebar[rc] : T(0);
#pragma unroll
            for (int sp = 0; sp < S; ++sp) wr[k][sp] = f.wsp[(size_t)sp * g.n_atm + rc];
        } else {
            rho[k] = (T)vc.albedo;
            Eb[k] = T(0);
#pragma unroll
            for (int sp = 0; sp < S; ++sp) wr[k][sp] = T(0);
        }
    }
    const T *tlen = tap_len<T>(gp);
    (void)tlen;
    for (int t = w; t < G.nt; t += W) {
        const ASlot &d = gp.aslot[G.t0 + t];
        const int4 a0 = __ldg(reinterpret_cast<const int4 *>(&d));
        const int4 a1 = __ldg(reinterpret_cast<const int4 *>(&d) + 1);
        const int4 a2 = __ldg(reinterpret_cast<const int4 *>(&d) + 2);
        const int src = a0.x, pre = a0.y, seg = a0.z, n1 = a0.w;
        const int aux = a1.x, tbase = a1.y, bits = a1.z, dir = a1.w;
        const int hgdir = a2.x, taps = a2.y, pre_off = a2.z, seg_off = a2.w;
        const int kind = bits & 15, bkind = (bits >> 4) & 15;
        const bool c_one = (bits >> 8) & 1, n1_ground = (bits >> 9) & 1, has_pre = (bits >> 10) & 1;
        const bool gsrc = (bits >> 11) & 1;
        const int pre_n = taps & 0xff, seg_n = (taps >> 8) & 0xff, hit_n = (taps >> 16) & 0xff;
        const T q = aslot_q<T>(d), dinv = aslot_dinv<T>(d), split = aslot_split<T>(d);
        const int hit_off = __ldg(&d.hit_off);
        T qsun[S];
#pragma unroll
        for (int sp = 0; sp < S; ++sp) qsun[sp] = !gsrc ? f.q_sun[sp * g.nd + dir] : T(0);
        T th[4] = {T(0), T(0), T(0), T(0)};
        if (!ground_row) {
#pragma unroll
            for (int sp = 0; sp < S; ++sp) {
                const T h = f.hgv[sp * ndir + hgdir];
#pragma unroll
                for (int k = 0; k < 4; ++k) th[k] += wr[k][sp] * h;
            }
        }
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            if (G.row[k] < 0) continue;
            const int rp = G.rp[k];
            const int j = rp + src;
            T tpre = T(0), tsg = T(0), thit = T(0);
            if (pre >= 0)
                tpre = __ldg(f.tseg + pre + rp);
            else if (pre_n)
                tpre = tap_sum_h<T>(gp, f.mu_e_h, pre_off, pre_n, rp + tbase);
            if (seg >= 0)
                tsg = __ldg(f.tseg + seg + rp);
            else if (seg_n)
                tsg = tap_sum_h<T>(gp, f.mu_e_h, seg_off, seg_n, rp + tbase);
            if (hit_n) thit = tap_sum_h<T>(gp, f.mu_e_h, hit_off, hit_n, rp + tbase);
            T Wi, Ws;
            if constexpr (kSel) {
                const size_t o = (size_t)dir * g.npad + j;
                Wi = __ldg(wsi + o);
                Ws = gsrc ? Wi : __ldg(wss + o);
            } else if (!gsrc) {
                T qs = T(0);
#pragma unroll
                for (int sp = 0; sp < S; ++sp) qs += __ldg(f.wsp_h + (size_t)sp * g.npad + j) * qsun[sp];
                T ci = T(1), cs = T(1);
                if (!c_one) {
                    const T rtn = n1_ground ? rt_lamb : __ldg(f.rt_h + rp + n1);
                    const T ai = __ldg(f.a_iso + j), as = __ldg(f.a_sun + j);
                    ci = ai > T(0) ? ai * rtn * dinv : T(1);
                    cs = as > T(0) ? as * rtn * dinv : T(1);
                }
                Wi = q * ci;
                Ws = qs * cs;
            } else {
                const T rtn = __ldg(f.rt_h + rp + n1);
                const T a = __ldg(f.a_iso + j);
                Wi = q * (a > T(0) ? a * rtn * dinv : T(1));
                Ws = Wi;
            }
            const T e1j = __ldg(f.e1_h + j);
            const T cc = lam[k] + Eb[k] * th[k];
            const T Y = (T)x64[j] * Wi + Ws * e1j;
            // P and dP/dtau for the slot's kind
            T P, gpre = T(0), gseg = T(0), gb = T(0), ghit = T(0);  // dP / dtau_*
            if (kind == 0 || kind == 3) {
                const T ep = has_pre ? fast_exp_neg<T>(tpre) : T(1);
                if (bkind == 0) {
                    P = ep * one_minus_exp<T>(tsg);
                    gseg = ep * fast_exp_neg<T>(tsg);
                } else if (bkind == 1) {
                    P = ep;
                } else {
                    const T tb = bkind == 2 ? f.tinf[(size_t)aux * g.n_atm + G.row[k]]
                                            : (bkind == 3 ? thit : __ldg(f.tinfg + aux + rp));
                    P = ep * one_minus_exp<T>(tsg + tb);
                    gseg = ep * fast_exp_neg<T>(tsg + tb);
                    gb = gseg;
                }
                if (has_pre) gpre = -P;
            } else if (kind == 1) {
                const T tb = bkind == 2 ? f.tinf[(size_t)aux * g.n_atm + G.row[k]] : thit;
                P = one_minus_exp<T>(tb);
                gb = fast_exp_neg<T>(tb);
            } else {
                P = split * fast_exp_neg<T>(tpre + thit);
                gpre = -P;
                ghit = -P;
            }
            rhob[k] += P * cc * Y;
            atomicAdd(ad.e1bar_h + j, cc * rho[k] * Ws * P);
            const T Pb = rho[k] * cc * Y;
            // optical depths back to their sources
            if (gpre != T(0)) {
                if (pre >= 0)
                    atomicAdd(ad.tsegbar + pre + rp, Pb * gpre);
                else
                    scatter_taps_h<T>(gp, pre_off, pre_n, rp + tbase, Pb * gpre, ad.mubar_h);
            }
            if (gseg != T(0)) {
                if (seg >= 0)
                    atomicAdd(ad.tsegbar + seg + rp, Pb * gseg);
                else
                    scatter_taps_h<T>(gp, seg_off, seg_n, rp + tbase, Pb * gseg, ad.mubar_h);
            }
            if (gb != T(0)) {
                const int bk = kind == 1 ? (bkind == 2 ? 2 : 3) : bkind;
                if (bk == 2)
                    atomicAdd(ad.tinfbar + (size_t)aux * g.n_atm + G.row[k], Pb * gb);
                else if (bk == 3)
                    scatter_taps_h<T>(gp, hit_off, hit_n, rp + tbase, Pb * gb, ad.mubar_h);
                else
                    atomicAdd(ad.tinfgbar + aux + rp, Pb * gb);
            }
            if (ghit != T(0)) scatter_taps_h<T>(gp, hit_off, hit_n, rp + tbase, Pb * ghit, ad.mubar_h);
        }
    }
    // rho_i = mu_s / mu_e:  mu_e-bar_i -= rho-bar_i rho_i / mu_e_i
#pragma unroll
    for (int k = 0; k < 4; ++k) sh[w][k][lane] = rhob[k];
    __syncthreads();
    if (w == 0 && !ground_row) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (G.row[k] < 0) continue;
            T rb = T(0);
#pragma unroll
            for (int qq = 0; qq < W; ++qq) rb += sh[qq][k][lane];
            const T me = f.mu_e[G.row[k]];
            if (me > T(0)) atomicAdd(ad.mubar + G.row[k], -rb * rho[k] / me);
        }
    }
}

// tau_inf(z) = tseg(node z going up) + tau_inf(z + dz) down each upward line,
// started from taps at the top: tseg-bar(node) = sum of tau_inf-bar at and
// below the node, the top taps get the sum of the whole line.
template <typename T>
__global__ void k_tinf_adj(GridC g, GraphP gp, FieldP<T> f, AdjP<T> ad) {
    const int ui = blockIdx.y, rem = blockIdx.x * blockDim.x + threadIdx.x;
    if (rem >= g.R * g.nxy) return;
    const int o = rem / g.nxy, c = rem - o * g.nxy;
    const int u = gp.up_dirs[ui];
    const int4 d = gp.dirs[u];
    if (o >= d.z) return;
    const int zt = g.nz - 1 - o;
    if (zt < 0) return;
    const int y0 = c / g.nx, x0 = c - y0 * g.nx;
    const int tab = gp.up_canon[ui];
    const T *tb = ad.tinfbar + (size_t)ui * g.n_atm;
    T acc = T(0);
    for (int s = zt / d.z; s >= 1; --s) {
        const int z = zt - s * d.z, x = wrap_any(x0 - s * d.x, g.nx), y = wrap_any(y0 - s * d.y, g.ny);
        acc += tb[(z * g.ny + y) * g.nx + x];
        if (acc != T(0)) atomicAdd(ad.tsegbar + (size_t)tab * g.npad + halo_pos(g, x, y, z), acc);
    }
    acc += tb[(zt * g.ny + y0) * g.nx + x0];
    scatter_taps<T>(g, gp.taps, tap_len<T>(gp), gp.top_off[ui * g.R + o], gp.top_n[ui * g.R + o], x0, y0, zt, acc,
                    ad.mubar);
}

// segment table entries back to the extinction along their lattice taps
template <typename T>
__global__ void k_tseg_adj(GridC g, GraphP gp, FieldP<T> f, AdjP<T> ad) {
    const int c = blockIdx.y, a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= g.n_atm) return;
    const int u = gp.canon_dirs[c];
    const int4 d = gp.dirs[u];
    const int z = a / g.nxy, r = a - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    if (z + d.z >= g.nz) return;
    const T tbar = gather_halo(ad.tsegbar + (size_t)c * g.npad, g, x, y, z);
    scatter_taps<T>(g, gp.taps, tap_len<T>(gp), gp.lat_off[u], gp.lat_n[u], x, y, z, tbar, ad.mubar);
}

// optical depths from the ground chains' last members to the TOA
template <typename T>
__global__ void k_tinfg_adj(GridC g, GraphP gp, FieldP<T> f, AdjP<T> ad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ngd * g.nxy) return;
    const int gd = t / g.nxy, c = t - gd * g.nxy;
    const int y = c / g.nx, x = c - y * g.nx;
    const T tbar = gather_halo(ad.tinfgbar + (size_t)gd * g.lp, g, x, y, 0);
    scatter_taps<T>(g, gp.taps, tap_len<T>(gp), gp.gtop_off[gd], gp.gtop_n[gd], x, y, 0, tbar, ad.mubar);
}

// e1: e1-bar from the pixels, the emission (e1_i theta0_i) and the slots;
// e1_i = omega_i B T_sun,i (1 - exp(-mu_e,i a)), a = hz / mu0 (atmosphere),
// e1_c = A B T_sun,c (ground); T_sun = exp(-tau_sun) along the sun taps.
template <typename T>
__global__ void k_e1_adj(GridC g, FieldP<T> f, ViewC vc, ViewP vp, AdjP<T> ad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_nodes) return;
    const int z = i / g.nxy, r = i - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    const bool atm = i < g.n_atm;
    T eb = ad.e1bar[i] + gather_halo(ad.e1bar_h, g, x, y, atm ? z : g.nz);
    if (atm) {
        T th0 = T(0);
        for (int sp = 0; sp < g.S; ++sp) th0 += f.wsp[(size_t)sp * g.n_atm + i] * f.hg0v[sp];
        eb += ad.Ebar[i] * th0;
    }
    if (eb == T(0)) return;
    const T e1 = f.e1[i];
    if (atm) {
        const T me = f.mu_e[i];
        if (me > T(0)) {
            const T a = (T)(g.hz / vc.mu0);
            const T B = (T)(vc.f0 * vc.mu0 * g.hx * g.hy);
            const T om = f.mu_st[i] / me;
            const T direct = -e1 / me + om * B * f.tsun[i] * a * dexp<T>(-me * a);
            atomicAdd(ad.mubar + i, eb * direct);
        }
    }
    const int Zs = atm ? z + 1 : 0;
    const T *len;
    if constexpr (sizeof(T) == 4)
        len = (const T *)vp.sun_len_f;
    else
        len = (const T *)vp.sun_len_d;
    scatter_taps<T>(g, vp.sun_taps, len, vp.sun_off[Zs], vp.sun_n[Zs], x, y, 0, -eb * e1, ad.mubar);
}

// mu_e-bar += the tap contributions accumulated in the haloed layout
template <typename T>
__global__ void k_mubar_gather(GridC g, AdjP<T> ad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_atm) return;
    const int z = i / g.nxy, r = i - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    ad.mubar[i] += gather_halo(ad.mubar_h, g, x, y, z);
}

// ---------------------------------------------------------------------------
// launchers

template <typename T>
void launch_transpose_vals(cudaStream_t st, const GridC &g, const GraphP &gp, const TransP &tp, const T *val,
                           T *valT) {
    k_transpose_vals<T><<<(g.nz + 1) * g.gpl, 256, 0, st>>>(g, gp, tp, val, valT);
}

template <typename T>
void launch_pix_adj(cudaStream_t st, const GridC &g, const FieldP<T> &f, const ViewC &vc, const ViewP &vp,
                    const T *emis, const double *x, const T *Lbar, const AdjP<T> &ad) {
    const long long n = (long long)vp.npx * vp.npy * 32;
    k_pix_adj<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, f, vc, vp, emis, x, Lbar, ad);
}

template <typename T>
void launch_emis_adj(cudaStream_t st, const GridC &g, const GraphP &gpT, const TransP &tp, const FieldP<T> &f,
                     const T *valT, const AdjP<T> &ad) {
    GridC g1 = g;
    g1.stage = 0;  // the transposed templates have no streamed runs
    auto go = [&](auto sp) {
        constexpr int S = decltype(sp)::value;
        OpEmisT<T, S> op;
        op.Ebar_h = ad.Ebar_h;
        op.wsp_h = f.wsp_h;
        op.hgv = f.hgv;
        op.hgdirT = tp.hgdir;
        op.xbar = ad.xbar;
        op.npad = g.npad;
        op.ndir = g.nd + g.ngd;
        run_op(st, g1, gpT, valT, op, 0);
    };
    switch (g.S) {
        case 1: go(std::integral_constant<int, 1>()); break;
        case 2: go(std::integral_constant<int, 2>()); break;
        case 3: go(std::integral_constant<int, 3>()); break;
        default: go(std::integral_constant<int, 4>()); break;
    }
}

template <typename T>
void launch_asm_adj(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                    const double *x64, const double *lam64, const AdjP<T> &ad) {
    const int nb = (g.nz + 1) * g.gpl;
    switch (g.S) {
        case 1: k_asm_adj<T, 1, false><<<nb, 32 * kAdjW, 0, st>>>(g, gp, f, vc, x64, lam64, ad, nullptr, nullptr); break;
        case 2: k_asm_adj<T, 2, false><<<nb, 32 * kAdjW, 0, st>>>(g, gp, f, vc, x64, lam64, ad, nullptr, nullptr); break;
        case 3: k_asm_adj<T, 3, false><<<nb, 32 * kAdjW, 0, st>>>(g, gp, f, vc, x64, lam64, ad, nullptr, nullptr); break;
        default: k_asm_adj<T, 4, false><<<nb, 32 * kAdjW, 0, st>>>(g, gp, f, vc, x64, lam64, ad, nullptr, nullptr); break;
    }
}

template <typename T>
void launch_asm_adj_sel(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                        const double *x64, const double *lam64, const AdjP<T> &ad, const T *w_iso,
                        const T *w_sun) {
    const int nb = (g.nz + 1) * g.gpl;
    switch (g.S) {
        case 1: k_asm_adj<T, 1, true><<<nb, 32 * kAdjW, 0, st>>>(g, gp, f, vc, x64, lam64, ad, w_iso, w_sun); break;
        case 2: k_asm_adj<T, 2, true><<<nb, 32 * kAdjW, 0, st>>>(g, gp, f, vc, x64, lam64, ad, w_iso, w_sun); break;
        case 3: k_asm_adj<T, 3, true><<<nb, 32 * kAdjW, 0, st>>>(g, gp, f, vc, x64, lam64, ad, w_iso, w_sun); break;
        default: k_asm_adj<T, 4, true><<<nb, 32 * kAdjW, 0, st>>>(g, gp, f, vc, x64, lam64, ad, w_iso, w_sun); break;
    }
}

template <typename T>
void launch_tables_adj(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                       const ViewP &vp, const AdjP<T> &ad) {
    const int th = 256;
    k_tinf_adj<T><<<dim3((g.R * g.nxy + th - 1) / th, g.nup), th, 0, st>>>(g, gp, f, ad);
    k_tseg_adj<T><<<dim3((g.n_atm + th - 1) / th, g.nc), th, 0, st>>>(g, gp, f, ad);
    k_tinfg_adj<T><<<(g.ngd * g.nxy + th - 1) / th, th, 0, st>>>(g, gp, f, ad);
    k_e1_adj<T><<<(g.n_nodes + th - 1) / th, th, 0, st>>>(g, f, vc, vp, ad);
    k_mubar_gather<T><<<(g.n_atm + th - 1) / th, th, 0, st>>>(g, ad);
}

#define INST(T)                                                                                                  \
    template void launch_transpose_vals<T>(cudaStream_t, const GridC &, const GraphP &, const TransP &,          \
                                           const T *, T *);                                                     \
    template void launch_pix_adj<T>(cudaStream_t, const GridC &, const FieldP<T> &, const ViewC &,              \
                                    const ViewP &, const T *, const double *, const T *, const AdjP<T> &);      \
    template void launch_emis_adj<T>(cudaStream_t, const GridC &, const GraphP &, const TransP &,               \
                                     const FieldP<T> &, const T *, const AdjP<T> &);                           \
    template void launch_asm_adj<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,             \
                                    const ViewC &, const double *, const double *, const AdjP<T> &);            \
    template void launch_asm_adj_sel<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,         \
                                        const ViewC &, const double *, const double *, const AdjP<T> &,         \
                                        const T *, const T *);                                                  \
    template void launch_tables_adj<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,          \
                                       const ViewC &, const ViewP &, const AdjP<T> &);
INST(float)
INST(double)
#undef INST

}  // namespace tk
