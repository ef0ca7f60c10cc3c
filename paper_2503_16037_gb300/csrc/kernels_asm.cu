// Assembly of the flux matrix K (rows = receivers), the direct solar source
// e1 and s = K^sun e1 on the GPU.
//
// Paper correspondence (Mikkonen et al., scattering graph method):
//   edge transmittance  exp(-int mu_e)         Eq. radiance_effectuality, Eq. Fab
//   quadrature weight   p' over a lattice cell Eq. F_term_phase, Sec. 3 (Fibonacci lattice)
//   coupling            C = sqrt(mu_s mu_s')/d Eq. scatt_coup (normalised routing weight)
//   external source     S_a                    Sec. 2 (far-field source)
// The deposit of a chain on its nodes lumps the extinction beyond the
// stencil on the terminal node; escape to the TOA leaves the graph.
//
// Layout: all receiver rows of one layer share a slot template, so the edge
// kernel runs one thread per row and a warp walks the template in lockstep:
// the slot class, its tap offsets and the chain kind are warp-uniform, the
// extinction gathers of a tap are coalesced along x, and the values are
// stored slot-major (val[voff + t * nxy + r]) with coalesced writes.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kern.h"
#include "stage.cuh"
#include "asm_util.cuh"
#include "first_order.h"
#include "select.h"
#include "aniso.h"

namespace tk {

// ---------------------------------------------------------------------------
// CSR export (row order = template order): one thread per row

template <typename T>
__global__ void k_export_csr(GridC g, GraphP gp, const T *__restrict__ val, int32_t *row_ptr, int32_t *col,
                             T *cval, int16_t *dir, int8_t *kk) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= g.n_nodes) return;
    int z = row / g.nxy, r = row - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    int t0 = gp.tstart[z], nt = gp.tstart[z + 1] - t0;
    // CSR offsets: all rows of earlier layers, then earlier rows of this layer
    long long e0 = 0;
    for (int zz = 0; zz < z; ++zz) e0 += (long long)(gp.tstart[zz + 1] - gp.tstart[zz]) * g.nxy;
    e0 += (long long)r * nt;
    const long long vb = val_base(gp.voff[z], nt, r);
    if (row_ptr) {
        row_ptr[row] = (int32_t)e0;
        if (row == g.n_nodes - 1) row_ptr[g.n_nodes] = (int32_t)(e0 + nt);
    }
    for (int t = 0; t < nt; ++t) {
        int4 te = gp.tmpl[t0 + t];
        const DClass &c = gp.cls[te.x];
        if (col) col[e0 + t] = slot_src(g, row, x, y, te);
        if (cval) cval[e0 + t] = val[vb + (long long)t * kGroup];
        if (dir) dir[e0 + t] = c.hgdir;
        if (kk) kk[e0 + t] = (int8_t)(c.kind == 1 ? 0 : c.kind == 2 ? 7 : c.k);
    }
}

template <typename T>
void launch_export_csr(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, int32_t *row_ptr,
                       int32_t *col, T *cval, int16_t *dir, int8_t *k) {
    k_export_csr<T><<<(g.n_nodes + 127) / 128, 128, 0, st>>>(g, gp, val, row_ptr, col, cval, dir, k);
}

// ---------------------------------------------------------------------------
// Field preparation: total scattering, extinction, validity, max mu_s

template <typename T>
__global__ void k_prep(GridC g, FieldP<T> f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (i < g.n_atm) {
        T a = f.mu_a[i];
        bool ok = isfinite((double)a) && a >= T(0);
        T s = T(0);
        #pragma unroll
        for (int sp = 0; sp < MAX_SPECIES; ++sp) if (sp < g.S) {
            T v = f.mu_s[(size_t)sp * g.n_atm + i];
            ok = ok && isfinite((double)v) && v >= T(0);
            s += v;
        }
        if (!ok) {
            atomicOr(f.status, STATUS_BAD_FIELD);
            s = T(0);
            a = T(0);
        }
        const int z = i / g.nxy, r = i - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
        f.mu_st[i] = s;
        f.mu_e[i] = a + s;
        store_halo(f.mu_e_h, g, x, y, z, a + s);
        const T rs = dsqrt<T>(s);
        f.rt[i] = rs;
        store_halo(f.rt_h, g, x, y, z, rs);
        T inv = s > T(0) ? T(1) / s : T(0);
        #pragma unroll
        for (int sp = 0; sp < MAX_SPECIES; ++sp) if (sp < g.S) {
            const T wv = s > T(0) ? f.mu_s[(size_t)sp * g.n_atm + i] * inv : T(1) / (T)g.S;
            f.wsp[(size_t)sp * g.n_atm + i] = wv;
            store_halo(f.wsp_h + (size_t)sp * g.npad, g, x, y, z, wv);
        }
        m = (double)s;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(f.mus_max_bits, (unsigned long long)__double_as_longlong(m));
}

// ---------------------------------------------------------------------------
// Quadrature tables of the scene geometry.  q^sun of species s and direction
// u is the HG-weighted fraction of the Fibonacci lattice in the cell of u;
// the sums are FP64 in a fixed order (one block per (cell, species)).

template <typename T>
__global__ void k_tables_cells(GridC g, FieldP<T> f, ViewC vc, ViewP vp) {
    __shared__ double red[32];
    int u = blockIdx.x, sp = blockIdx.y;
    double gg = sp == 0 ? vc.g[0] : sp == 1 ? vc.g[1] : sp == 2 ? vc.g[2] : vc.g[3];
    double acc = 0.0;
    for (int m = vp.cell_start[u] + threadIdx.x; m < vp.cell_start[u + 1]; m += blockDim.x) {
        const double *s = vp.lattice + 3 * (size_t)m;
        double mu = vc.s0[0] * s[0] + vc.s0[1] * s[1] + vc.s0[2] * s[2];
        acc += hg<double>(gg, mu);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        f.cellsum[sp * g.nd + u] = t;
    }
}

template <typename T>
__global__ void k_tables_norm(GridC g, FieldP<T> f, ViewC vc, ViewP vp) {
    __shared__ double total;
    int sp = blockIdx.x;
    double gg = sp == 0 ? vc.g[0] : sp == 1 ? vc.g[1] : sp == 2 ? vc.g[2] : vc.g[3];
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int u = 0; u < g.nd; ++u) t += f.cellsum[sp * g.nd + u];
        total = t;
    }
    __syncthreads();
    for (int u = threadIdx.x; u < g.nd; u += blockDim.x) f.q_sun[sp * g.nd + u] = (T)(f.cellsum[sp * g.nd + u] / total);
    int ndir = g.nd + g.ngd;
    for (int d = threadIdx.x; d < ndir; d += blockDim.x) {
        const double *h = vp.dirhat + 3 * d;
        double mu = h[0] * vc.v[0] + h[1] * vc.v[1] + h[2] * vc.v[2];
        f.hgv[sp * ndir + d] = (T)hg<double>(gg, mu);
    }
    if (threadIdx.x == 0) {
        double mu = vc.s0[0] * vc.v[0] + vc.s0[1] * vc.v[1] + vc.s0[2] * vc.v[2];
        f.hg0v[sp] = (T)hg<double>(gg, mu);
    }
}

// ---------------------------------------------------------------------------
// Direct beam: transmittance from the TOA to each voxel's top-face centre
// (ground point for ground nodes) and the first-order scattered power
//   e1_j = omega_j f0 mu0 hx hy T_sun (1 - exp(-mu_e hz / mu0)),
//   e1_c = A f0 mu0 hx hy T_sun.

template <typename T>
__global__ void k_sun(GridC g, FieldP<T> f, ViewC vc, ViewP vp) {
    // kRayLanes lanes per node; lanes past the last node work on the last
    // node and write nothing (they take part in the group's shuffles)
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const bool own = gt / kRayLanes < g.n_nodes && (threadIdx.x & (kRayLanes - 1)) == 0;
    const int i = min(gt / kRayLanes, g.n_nodes - 1);
    int z = i / g.nxy, r = i - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    int Zs = i < g.n_atm ? z + 1 : 0;
    const T *len;
    if constexpr (sizeof(T) == 4)
        len = (const T *)vp.sun_len_f;
    else
        len = (const T *)vp.sun_len_d;
    T tau = ray_sum_lanes<T>(g, vp.sun_rt, len, f.mu_e, __ldg(vp.sun_off + Zs), __ldg(vp.sun_n + Zs), x, y);
    if (!own) return;
    T Ts = dexp<T>(-tau);
    f.tsun[i] = Ts;
    T base = (T)(vc.f0 * vc.mu0 * g.hx * g.hy);
    if (i < g.n_atm) {
        T me = f.mu_e[i];
        T om = me > T(0) ? f.mu_st[i] / me : T(0);
        const T e = om * base * Ts * (-dexpm1<T>(-me * (T)(g.hz / vc.mu0)));
        f.e1[i] = e;
        store_halo(f.e1_h, g, x, y, z, e);
    } else {
        const T e = (T)vc.albedo * base * Ts;
        f.e1[i] = e;
        store_halo(f.e1_h, g, x, y, g.nz, e);
    }
}

// ---------------------------------------------------------------------------
// Optical depth of the lattice segment from every voxel centre a to a + u, for
// each canonical direction u (one of each pair {u, -u}); a segment traversed
// backwards (-u, from a + u) reads the same entry.  One thread per voxel a
// walks kSegChunk directions (blockIdx.y: the chunk), so its coordinates and
// halo copies are worked out once per chunk; entries whose end lies above the
// TOA are not used and are set to 0.
constexpr int kSegChunk = 7;

template <typename T>
__global__ void k_segtau(GridC g, GraphP gp, FieldP<T> f) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= g.n_atm) return;
    const int z = a / g.nxy, r = a - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    const int p = (int)halo_pos(g, x, y, z);
    const int ax = x < g.H ? g.nx : (x >= g.nx - g.H ? -g.nx : 0);
    const int ay = y < g.H ? g.ny * g.nxp : (y >= g.ny - g.H ? -g.ny * g.nxp : 0);
    const int c1 = min((int)(blockIdx.y + 1) * kSegChunk, g.nc);
    for (int c = blockIdx.y * kSegChunk; c < c1; ++c) {
        const int u = __ldg(gp.canon_dirs + c);
        T tau = T(0);
        if (z + __ldg(&gp.dirs[u].z) < g.nz) tau = tap_sum_h<T>(gp, f.mu_e_h, __ldg(gp.lat_off + u), __ldg(gp.lat_n + u), p);
        T *o = f.tseg + (size_t)c * g.npad + p;
        o[0] = tau;
        if (ax) o[ax] = tau;
        if (ay) {
            o[ay] = tau;
            if (ax) o[ax + ay] = tau;
        }
    }
}


// Optical depth from each voxel centre to the TOA along each upward lattice
// direction, by recursion down the lattice lines:
//   tau_inf(j, u) = tau(j -> j + u) + tau_inf(j + u, u).
// One thread per (upward direction, start layer offset, column).
template <typename T>
__global__ void k_tinf(GridC g, GraphP gp, FieldP<T> f) {
    const int ui = blockIdx.y, rem = blockIdx.x * blockDim.x + threadIdx.x;
    if (rem >= g.R * g.nxy) return;
    const int o = rem / g.nxy, c = rem - o * g.nxy;
    int u = gp.up_dirs[ui];
    int4 d = gp.dirs[u];
    if (o >= d.z) return;
    int zt = g.nz - 1 - o;
    if (zt < 0) return;
    int y = c / g.nx, x = c - y * g.nx;
    T tau = tap_sum<T>(g, gp, f.mu_e, gp.top_off[ui * g.R + o], gp.top_n[ui * g.R + o], x, y, zt);
    T *out = f.tinf + (size_t)ui * g.n_atm;
    out[(zt * g.ny + y) * g.nx + x] = tau;
    const int tab = gp.up_canon[ui];
    for (int z = zt - d.z; z >= 0; z -= d.z) {
        x = wrap_small(x - d.x, g.nx);
        y = wrap_small(y - d.y, g.ny);
        tau += seg_at<T>(g, f.tseg, tab, x, y, z);
        out[(z * g.ny + y) * g.nx + x] = tau;
    }
}

// ground chains: optical depth from the terminal member to the TOA
// (kRayLanes lanes per ray, as in k_sun)
template <typename T>
__global__ void k_tinfg(GridC g, GraphP gp, FieldP<T> f) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const bool own = gt / kRayLanes < g.ngd * g.nxy && (threadIdx.x & (kRayLanes - 1)) == 0;
    const int t = min(gt / kRayLanes, g.ngd * g.nxy - 1);
    int gd = t / g.nxy, c = t - gd * g.nxy;
    int y = c / g.nx, x = c - y * g.nx;
    const T tau = ray_sum_lanes<T>(g, gp.rtaps, tap_len<T>(gp), f.mu_e, __ldg(gp.gtop_off + gd), __ldg(gp.gtop_n + gd), x, y);
    // haloed plane of ground direction gd: layer index 0 of a (1 x lp) array
    if (own) store_halo(f.tinfg + (size_t)gd * g.lp, g, x, y, 0, tau);
}

// ---------------------------------------------------------------------------
// Coupling normalisers (Eq. scatt_coup as a routing weight): for each source
//   zc = sum_{U_c} q / sum_{U_c} q C   (0 when the coupling is off or the
// denominator vanishes), so that c_{j,u} = C_{j,u} zc and sum_u q c = 1,
// with C_{j,u} = sqrt(mu_s(j)) sqrt(mu_s(n1)) / d.  U_c: directions whose
// chain has a receiver other than the source.

template <typename T>
__global__ void k_znorm(GridC g, GraphP gp, FieldP<T> f, ViewC vc) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_nodes) return;
    const T rt_lamb = dsqrt<T>((T)(vc.albedo * __longlong_as_double((long long)*f.mus_max_bits)));
    T sq_i = 0, sqc_i = 0, sq_s = 0, sqc_s = 0;
    int z = j / g.nxy, r = j - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    T rt_src;
    if (j < g.n_atm) {
        rt_src = f.rt[j];
        const T *rt_j = f.rt_h + halo_pos(g, x, y, z);  // |u_x|, |u_y| <= R: no wrap
        T w[MAX_SPECIES];
        #pragma unroll
        for (int sp = 0; sp < MAX_SPECIES; ++sp) if (sp < g.S) w[sp] = f.wsp[(size_t)sp * g.n_atm + j];
#pragma unroll 4
        for (int u = 0; u < g.nd; ++u) {
            int4 d = gp.dirs[u];
            int rz = z + d.z;
            T rtn, dist;
            if (rz >= 0 && rz < g.nz) {
                rtn = __ldg(rt_j + __ldg(gp.dir_h + u));
                dist = Cst<T>::dir_len(gp, u);
            } else if (d.z < 0) {
                rtn = rt_lamb;
                dist = ((T)z + T(0.5)) / (T)(-d.z) * Cst<T>::dir_len(gp, u);
            } else {
                continue;
            }
            T C = rt_src * rtn / dist;
            T qi = Cst<T>::q_iso(gp, u);
            T qs = T(0);
            #pragma unroll
            for (int sp = 0; sp < MAX_SPECIES; ++sp) if (sp < g.S) qs += w[sp] * f.q_sun[sp * g.nd + u];
            sq_i += qi;
            sqc_i += qi * C;
            sq_s += qs;
            sqc_s += qs * C;
        }
    } else {
        rt_src = rt_lamb;
        for (int gd = 0; gd < g.ngd; ++gd) {
            int4 m = gp.gmem1[gd];
            T rtn = f.rt[((m.z - 1) * g.ny + wrap_small(y + m.y, g.ny)) * g.nx + wrap_small(x + m.x, g.nx)];
            T C = rt_src * rtn / Cst<T>::gdist1(gp, gd);
            T q = Cst<T>::q_lamb(gp, gd);
            sq_i += q;
            sqc_i += q * C;
        }
        sq_s = sq_i;
        sqc_s = sqc_i;
    }
    // stored premultiplied by sqrt(mu_s) of the source: c = a sqrt(mu_s(n1)) / d
    const int zz = j < g.n_atm ? z : g.nz;
    store_halo(f.a_iso, g, x, y, zz, (vc.coupling && sqc_i > T(0)) ? sq_i / sqc_i * rt_src : T(0));
    store_halo(f.a_sun, g, x, y, zz, (vc.coupling && sqc_s > T(0)) ? sq_s / sqc_s * rt_src : T(0));
}

// ---------------------------------------------------------------------------
// Fused edge march + edge weights, one block of kAsmW warps per group of 128
// receiver rows (lane l owns rows l + 32k; warp w takes the slots t = w mod
// kAsmW).  For every slot the optical depths of the chain segments come from
// the per-node segment table (or, for partial segments, from tap lists over
// the extinction), the deposit fraction P, the quadrature weight q and the
// coupling c of the source give
//   K_ij = rho_i q_{j,u} c_{j,u} P          (stored slot-major per group)
//   s_i  = sum_slots rho_i q^sun c^sun P e1_j
//   g_i  = sum_slots Theta_i(u . v) rho_i q^sun c^sun P e1_j   (atmospheric rows)
// Every lookup is one add from the receiver's haloed position (the slot's
// ASlot descriptor holds the offsets), so a warp's loads of one slot cover
// contiguous lines.
// warps per group and the register budget (blocks per SM): measured best on
// GB300 at 8 warps and 4 blocks (64 registers)
#ifndef TK_ASM_W
#define TK_ASM_W 8
#endif
constexpr int kAsmW = TK_ASM_W;

#ifndef TK_ASM_MINB
#define TK_ASM_MINB 4
#endif
// kMode 0: K.  kMode 1 (coupling selection): K with the weights q c of every
// (source, direction) read from the planes wsi / wss (haloed, one per
// direction) instead of the global quadrature and the source's normaliser.
// kMode 2 (anisotropic multiple scattering): the raw deposit fraction P of
// every slot instead of K (s and g^sun as in mode 0).
template <typename T, int S, int kMode>
__global__ void __launch_bounds__(32 * kAsmW, TK_ASM_MINB)
    k_asm(GridC g, GraphP gp, FieldP<T> f, ViewC vc, const T *__restrict__ wsi, const T *__restrict__ wss) {
    __shared__ T sh[kAsmW][8][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const GroupRows G = group_rows(g, gp, blockIdx.x);
    const bool ground_row = G.z == g.nz;
    const T rt_lamb = dsqrt<T>((T)(vc.albedo * __longlong_as_double((long long)*f.mus_max_bits)));
    const int ndir = g.nd + g.ngd;
    int rowc[4];
    T rho[4], wr[4][S];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        rowc[k] = G.row[k] >= 0 ? G.row[k] : G.z * g.nxy;  // rows past the layer's end read a valid node
        if (!ground_row) {
            const T me = f.mu_e[rowc[k]], ms = f.mu_st[rowc[k]];
            rho[k] = me > T(0) ? ms / me : T(0);
#pragma unroll
            for (int sp = 0; sp < S; ++sp) wr[k][sp] = f.wsp[(size_t)sp * g.n_atm + rowc[k]];
        } else {
            rho[k] = (T)vc.albedo;
#pragma unroll
            for (int sp = 0; sp < S; ++sp) wr[k][sp] = T(0);
        }
    }
    T acc_s[4] = {T(0), T(0), T(0), T(0)}, acc_g[4] = {T(0), T(0), T(0), T(0)};
    T *vout = f.val + G.vb + 4 * lane;
    for (int t = w; t < G.nt; t += kAsmW) {
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
        T kv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
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
            T P;
            if (kind == 0 || kind == 3) {  // chain node (atmospheric or ground source)
                const T ep = has_pre ? fast_exp_neg<T>(tpre) : T(1);
                if (bkind == 0) {
                    P = ep * one_minus_exp<T>(tsg);
                } else if (bkind == 1) {
                    P = ep;
                } else {
                    const T tb = bkind == 2 ? f.tinf[(size_t)aux * g.n_atm + rowc[k]]
                                            : (bkind == 3 ? thit : __ldg(f.tinfg + aux + rp));
                    P = ep * one_minus_exp<T>(tsg + tb);
                }
            } else if (kind == 1) {  // self deposit
                const T tb = bkind == 2 ? f.tinf[(size_t)aux * g.n_atm + rowc[k]] : thit;
                P = one_minus_exp<T>(tb);
            } else {  // ground hit
                P = split * fast_exp_neg<T>(tpre + thit);
            }
            T Wi, Ws;
            if constexpr (kMode == 1) {
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
            kv[k] = kMode == 2 ? P : rho[k] * Wi * P;
            const T sun = rho[k] * Ws * P * __ldg(f.e1_h + j);
            acc_s[k] += sun;
            acc_g[k] += th[k] * sun;
        }
        st_quad(vout + (size_t)t * kGroup, kv);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        sh[w][k][lane] = acc_s[k];
        sh[w][4 + k][lane] = acc_g[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (G.row[k] < 0) continue;
            T a = T(0), b = T(0);
#pragma unroll
            for (int qq = 0; qq < kAsmW; ++qq) {
                a += sh[qq][k][lane];
                b += sh[qq][4 + k][lane];
            }
            f.s[G.row[k]] = a;
            if (!ground_row) f.gsun[G.row[k]] = b;
        }
    }
}

// Per-scene tables.  Dependencies: prep -> {sun, segtau -> tinf, tinfg, znorm};
// tables -> znorm.  st[0] is the scene stream; st[1..3] are auxiliary streams
// forked from it and joined back with events, so the independent tables run
// concurrently.
template <typename T>
void launch_assemble_pre(cudaStream_t const st[4], cudaEvent_t const ev[5], const GridC &g, const GraphP &gp,
                         const FieldP<T> &f, const ViewC &vc, const ViewP &vp, long long *launches) {
    const int th = 256;
    // ev[0]: start (orders the aux streams after earlier work of the scene stream)
    cudaEventRecord(ev[0], st[0]);
    cudaStreamWaitEvent(st[1], ev[0], 0);
    k_tables_cells<T><<<dim3(g.nd, g.S), 128, 0, st[1]>>>(g, f, vc, vp);
    k_tables_norm<T><<<g.S, 128, 0, st[1]>>>(g, f, vc, vp);
    cudaEventRecord(ev[2], st[1]);
    cudaMemsetAsync(f.mus_max_bits, 0, sizeof(unsigned long long), st[0]);
    k_prep<T><<<(g.n_atm + th - 1) / th, th, 0, st[0]>>>(g, f);
    cudaEventRecord(ev[1], st[0]);  // fields ready
    cudaStreamWaitEvent(st[2], ev[1], 0);
    k_segtau<T><<<dim3((g.n_atm + th - 1) / th, (g.nc + kSegChunk - 1) / kSegChunk), th, 0, st[2]>>>(g, gp, f);
    k_tinf<T><<<dim3((g.R * g.nxy + th - 1) / th, g.nup), th, 0, st[2]>>>(g, gp, f);
    cudaEventRecord(ev[3], st[2]);
    cudaStreamWaitEvent(st[3], ev[1], 0);
    k_tinfg<T><<<((long long)g.ngd * g.nxy * kRayLanes + 127) / 128, 128, 0, st[3]>>>(g, gp, f);
    k_sun<T><<<((long long)g.n_nodes * kRayLanes + 127) / 128, 128, 0, st[3]>>>(g, f, vc, vp);
    cudaEventRecord(ev[4], st[3]);
    cudaStreamWaitEvent(st[0], ev[2], 0);
    k_znorm<T><<<(g.n_nodes + 127) / 128, 128, 0, st[0]>>>(g, gp, f, vc);
    cudaStreamWaitEvent(st[0], ev[3], 0);
    cudaStreamWaitEvent(st[0], ev[4], 0);
    if (launches) *launches += 8;
}

template <typename T>
void launch_assemble_rows(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                          long long *launches) {
    const int nb = (g.nz + 1) * g.gpl;
    switch (g.S) {  // the species count as a compile-time constant
        case 1: k_asm<T, 1, 0><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, nullptr, nullptr); break;
        case 2: k_asm<T, 2, 0><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, nullptr, nullptr); break;
        case 3: k_asm<T, 3, 0><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, nullptr, nullptr); break;
        default: k_asm<T, 4, 0><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, nullptr, nullptr); break;
    }
    if (launches) *launches += 1;
}

template <typename T>
void launch_assemble_rows_sel(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f,
                              const ViewC &vc, const T *w_iso, const T *w_sun, long long *launches) {
    const int nb = (g.nz + 1) * g.gpl;
    switch (g.S) {
        case 1: k_asm<T, 1, 1><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, w_iso, w_sun); break;
        case 2: k_asm<T, 2, 1><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, w_iso, w_sun); break;
        case 3: k_asm<T, 3, 1><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, w_iso, w_sun); break;
        default: k_asm<T, 4, 1><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, w_iso, w_sun); break;
    }
    if (launches) *launches += 1;
}

template <typename T>
void launch_assemble_rows_p(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f,
                            const ViewC &vc, long long *launches) {
    const int nb = (g.nz + 1) * g.gpl;
    switch (g.S) {
        case 1: k_asm<T, 1, 2><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, nullptr, nullptr); break;
        case 2: k_asm<T, 2, 2><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, nullptr, nullptr); break;
        case 3: k_asm<T, 3, 2><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, nullptr, nullptr); break;
        default: k_asm<T, 4, 2><<<nb, 32 * kAsmW, 0, st>>>(g, gp, f, vc, nullptr, nullptr); break;
    }
    if (launches) *launches += 1;
}

// The first-order path: the phase tables, then the voxel fields and the
// direct beam, all on the scene stream (the edge tables are not needed).
template <typename T>
void launch_assemble_direct(cudaStream_t st, const GridC &g, const FieldP<T> &f, const ViewC &vc, const ViewP &vp,
                            long long *launches) {
    const int th = 256;
    k_tables_cells<T><<<dim3(g.nd, g.S), 128, 0, st>>>(g, f, vc, vp);
    k_tables_norm<T><<<g.S, 128, 0, st>>>(g, f, vc, vp);
    cudaMemsetAsync(f.mus_max_bits, 0, sizeof(unsigned long long), st);
    k_prep<T><<<(g.n_atm + th - 1) / th, th, 0, st>>>(g, f);
    k_sun<T><<<((long long)g.n_nodes * kRayLanes + 127) / 128, 128, 0, st>>>(g, f, vc, vp);
    if (launches) *launches += 4;
}

#define INST(T)                                                                                                   \
    template void launch_assemble_direct<T>(cudaStream_t, const GridC &, const FieldP<T> &, const ViewC &,       \
                                            const ViewP &, long long *);                                          \
    template void launch_assemble_rows_sel<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,     \
                                              const ViewC &, const T *, const T *, long long *);                  \
    template void launch_assemble_rows_p<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,       \
                                            const ViewC &, long long *);                                          \
    template void launch_assemble_pre<T>(cudaStream_t const[4], cudaEvent_t const[5], const GridC &,              \
                                         const GraphP &, const FieldP<T> &, const ViewC &, const ViewP &,         \
                                         long long *);                                                            \
    template void launch_assemble_rows<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,         \
                                          const ViewC &, long long *);                                            \
    template void launch_export_csr<T>(cudaStream_t, const GridC &, const GraphP &, const T *, int32_t *,         \
                                       int32_t *, T *, int16_t *, int8_t *);
INST(float)
INST(double)
#undef INST

}  // namespace tk
