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
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

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

template <typename T>
__device__ __forceinline__ const T *tap_len(const GraphP &gp);
template <>
__device__ __forceinline__ const float *tap_len<float>(const GraphP &gp) { return gp.tap_len_f; }
template <>
__device__ __forceinline__ const double *tap_len<double>(const GraphP &gp) { return gp.tap_len_d; }

__device__ __forceinline__ int wrap_small(int a, int n) {  // |a| < 2n
    a = a < 0 ? a + n : a;
    return a >= n ? a - n : a;
}
__device__ __forceinline__ int wrap_any(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// optical depth of a tap list based at cell (bx, by, bz); offsets small (stencil)
template <typename T>
__device__ __forceinline__ T tap_sum(const GridC &g, const GraphP &gp, const T *mu_e, int off, int n, int bx, int by,
                                     int bz) {
    const T *len = tap_len<T>(gp);
    T acc = T(0);
    for (int t = 0; t < n; ++t) {
        DTap tp = gp.taps[off + t];
        int x = wrap_small(bx + tp.dx, g.nx), y = wrap_small(by + tp.dy, g.ny), z = bz + tp.dz;
        acc += len[off + t] * mu_e[(z * g.ny + y) * g.nx + x];
    }
    return acc;
}

// same for long rays whose horizontal offsets may exceed the grid (any wrap)
template <typename T>
__device__ __forceinline__ T tap_sum_far(const GridC &g, const GraphP &gp, const T *mu_e, int off, int n, int bx,
                                         int by, int bz) {
    const T *len = tap_len<T>(gp);
    T acc = T(0);
    for (int t = 0; t < n; ++t) {
        DTap tp = gp.taps[off + t];
        int x = wrap_any(bx + tp.dx, g.nx), y = wrap_any(by + tp.dy, g.ny), z = bz + tp.dz;
        acc += len[off + t] * mu_e[(z * g.ny + y) * g.nx + x];
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ T hg(T g, T mu) {
    T d = T(1) + g * g - T(2) * g * mu;
    return (T(1) - g * g) / (T(4.0 * 3.14159265358979323846) * d * dsqrt<T>(d));
}

// ---------------------------------------------------------------------------
// CSR structure from the per-layer row templates (one warp per row)

__global__ void k_expand(GridC g, const int *tmpl_start, const int4 *tmpl, const int *tmpl_len, int32_t *row_ptr,
                         int32_t *col, uint16_t *code) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= g.n_nodes) return;
    int i = warp, z, x, y;
    if (i < g.n_atm) {
        z = i / g.nxy;
        int r = i - z * g.nxy;
        y = r / g.nx;
        x = r - y * g.nx;
    } else {
        z = g.nz;
        int r = i - g.n_atm;
        y = r / g.nx;
        x = r - y * g.nx;
    }
    // row start: all rows of earlier templates, then earlier rows of this layer
    long long e0 = 0;
    for (int zz = 0; zz < z; ++zz) e0 += (long long)tmpl_len[zz] * g.nxy;
    e0 += (long long)(i - (z < g.nz ? z * g.nxy : g.n_atm)) * tmpl_len[z];
    if (lane == 0) {
        row_ptr[i] = (int32_t)e0;
        if (i == g.n_nodes - 1) row_ptr[g.n_nodes] = (int32_t)(e0 + tmpl_len[z]);
    }
    int t0 = tmpl_start[z], n = tmpl_start[z + 1] - t0;
    for (int t = lane; t < n; t += 32) {
        int4 s = tmpl[t0 + t];  // (cls, sdx, sdy, sz)
        int sx = wrap_small(x + s.y, g.nx), sy = wrap_small(y + s.z, g.ny);
        int src = s.w >= 0 ? (s.w * g.ny + sy) * g.nx + sx : g.n_atm + sy * g.nx + sx;
        col[e0 + t] = src;
        code[e0 + t] = (uint16_t)s.x;
    }
}

void launch_expand(cudaStream_t st, const GridC &g, const int *tmpl_start, const int4 *tmpl, const int *tmpl_len,
                   int32_t *row_ptr, int32_t *col, uint16_t *code) {
    int threads = 256;
    long long blocks = ((long long)g.n_nodes * 32 + threads - 1) / threads;
    k_expand<<<(unsigned)blocks, threads, 0, st>>>(g, tmpl_start, tmpl, tmpl_len, row_ptr, col, code);
}

__global__ void k_slot_info(long long nnz, const uint16_t *code, const DClass *cls, int16_t *dir, int8_t *k, int nd) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const DClass &c = cls[code[e]];
    if (c.kind == 4) {
        dir[e] = -1;
        k[e] = -1;
    } else {
        dir[e] = c.hgdir;
        k[e] = (int8_t)(c.kind == 1 ? 0 : c.kind == 2 ? 7 : c.k);
    }
    (void)nd;
}

void launch_slot_info(cudaStream_t st, long long nnz, const uint16_t *code, const DClass *cls, int16_t *dir,
                      int8_t *k, int nd) {
    k_slot_info<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(nnz, code, cls, dir, k, nd);
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
        for (int sp = 0; sp < g.S; ++sp) {
            T v = f.mu_s[(size_t)sp * g.n_atm + i];
            ok = ok && isfinite((double)v) && v >= T(0);
            s += v;
        }
        if (!ok) {
            atomicOr(f.status, STATUS_BAD_FIELD);
            s = T(0);
            a = T(0);
        }
        f.mu_st[i] = s;
        f.mu_e[i] = a + s;
        m = (double)s;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0)
        atomicMax(f.mus_max_bits, (unsigned long long)__double_as_longlong(m));
}

// ---------------------------------------------------------------------------
// Quadrature tables of the scene geometry: q^sun per species and direction
// (HG-weighted Fibonacci cell fractions, FP64 sums in a fixed order), and the
// HG values toward the instrument for every travel direction.
// One block per species.

template <typename T>
__global__ void k_tables(GridC g, FieldP<T> f, ViewC vc, ViewP vp) {
    extern __shared__ double cellsum[];  // [nd]
    int sp = blockIdx.x;
    double gg = vc.g[sp];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int u = warp; u < g.nd; u += nw) {
        double acc = 0.0;
        for (int m = vp.cell_start[u] + lane; m < vp.cell_start[u + 1]; m += 32) {
            const double *s = vp.lattice + 3 * (size_t)m;
            double mu = vc.s0[0] * s[0] + vc.s0[1] * s[1] + vc.s0[2] * s[2];
            acc += hg<double>(gg, mu);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) cellsum[u] = acc;
    }
    __syncthreads();
    __shared__ double total;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int u = 0; u < g.nd; ++u) t += cellsum[u];
        total = t;
    }
    __syncthreads();
    for (int u = threadIdx.x; u < g.nd; u += blockDim.x) f.q_sun[sp * g.nd + u] = (T)(cellsum[u] / total);
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
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_nodes) return;
    int x, y, Zs;
    if (i < g.n_atm) {
        int z = i / g.nxy, r = i - z * g.nxy;
        y = r / g.nx;
        x = r - y * g.nx;
        Zs = z + 1;
    } else {
        int r = i - g.n_atm;
        y = r / g.nx;
        x = r - y * g.nx;
        Zs = 0;
    }
    const T *len = nullptr;
    if constexpr (sizeof(T) == 4)
        len = (const T *)vp.sun_len_f;
    else
        len = (const T *)vp.sun_len_d;
    int off = vp.sun_off[Zs], n = vp.sun_n[Zs];
    T tau = T(0);
    for (int t = 0; t < n; ++t) {
        DTap tp = vp.sun_taps[off + t];
        int xx = wrap_any(x + tp.dx, g.nx), yy = wrap_any(y + tp.dy, g.ny);
        tau += len[off + t] * f.mu_e[(tp.dz * g.ny + yy) * g.nx + xx];
    }
    T Ts = dexp<T>(-tau);
    f.tsun[i] = Ts;
    T base = (T)(vc.f0 * vc.mu0 * g.hx * g.hy);
    if (i < g.n_atm) {
        T me = f.mu_e[i];
        T om = me > T(0) ? f.mu_st[i] / me : T(0);
        f.e1[i] = om * base * Ts * (-dexpm1<T>(-me * (T)(g.hz / vc.mu0)));
    } else {
        f.e1[i] = (T)vc.albedo * base * Ts;
    }
}

// ---------------------------------------------------------------------------
// Optical depth from each voxel centre to the TOA along each upward lattice
// direction, by recursion down the lattice lines:
//   tau_inf(j, u) = tau(j -> j + u) + tau_inf(j + u, u).
// One thread per (upward direction, start layer offset, column).

template <typename T>
__global__ void k_tinf(GridC g, GraphP gp, FieldP<T> f) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long per = (long long)g.R * g.nxy;
    if (t >= per * g.nup) return;
    int ui = (int)(t / per);
    int rem = (int)(t - (long long)ui * per);
    int o = rem / g.nxy, c = rem - o * g.nxy;
    int u = gp.up_dirs[ui];
    int4 d = gp.dirs[u];
    if (o >= d.z) return;
    int zt = g.nz - 1 - o;
    if (zt < 0) return;
    int y = c / g.nx, x = c - y * g.nx;
    T tau = tap_sum<T>(g, gp, f.mu_e, gp.top_off[ui * g.R + o], gp.top_n[ui * g.R + o], x, y, zt);
    T *out = f.tinf + (size_t)ui * g.n_atm;
    out[(zt * g.ny + y) * g.nx + x] = tau;
    int loff = gp.lat_off[u], ln = gp.lat_n[u];
    for (int z = zt - d.z; z >= 0; z -= d.z) {
        x = wrap_small(x - d.x, g.nx);
        y = wrap_small(y - d.y, g.ny);
        tau += tap_sum<T>(g, gp, f.mu_e, loff, ln, x, y, z);
        out[(z * g.ny + y) * g.nx + x] = tau;
    }
}

// ground chains: optical depth from the terminal member to the TOA
template <typename T>
__global__ void k_tinfg(GridC g, GraphP gp, FieldP<T> f) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.ngd * g.nxy) return;
    int gd = t / g.nxy, c = t - gd * g.nxy;
    int y = c / g.nx, x = c - y * g.nx;
    f.tinfg[t] = tap_sum_far<T>(g, gp, f.mu_e, gp.gtop_off[gd], gp.gtop_n[gd], x, y, 0);
}

// ---------------------------------------------------------------------------
// Coupling normalisers (Eq. scatt_coup as a routing weight): for each source
//   zc = sum_{U_c} q / sum_{U_c} q C   (0 when the coupling is off or the
// denominator vanishes), so that c_{j,u} = C_{j,u} zc and sum_u q c = 1.
// U_c: directions whose chain has a receiver other than the source.

template <typename T>
__global__ void k_znorm(GridC g, GraphP gp, FieldP<T> f, ViewC vc) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_nodes) return;
    T mus_lamb = (T)(vc.albedo * __longlong_as_double((long long)*f.mus_max_bits));
    T sq_i = 0, sqc_i = 0, sq_s = 0, sqc_s = 0;
    if (j < g.n_atm) {
        int z = j / g.nxy, r = j - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
        T mus = f.mu_st[j];
        T w[MAX_SPECIES];
        for (int sp = 0; sp < g.S; ++sp)
            w[sp] = mus > T(0) ? f.mu_s[(size_t)sp * g.n_atm + j] / mus : T(1) / (T)g.S;
        for (int u = 0; u < g.nd; ++u) {
            int4 d = gp.dirs[u];
            int rz = z + d.z;
            T mun, dist;
            if (rz >= 0 && rz < g.nz) {
                mun = f.mu_st[(rz * g.ny + wrap_small(y + d.y, g.ny)) * g.nx + wrap_small(x + d.x, g.nx)];
                dist = (T)gp.dir_len[u];
            } else if (d.z < 0) {
                mun = mus_lamb;
                dist = (T)((z + 0.5) / (double)(-d.z) * gp.dir_len[u]);
            } else {
                continue;
            }
            T C = dsqrt<T>(mus * mun) / dist;
            T qi = (T)gp.q_iso[u];
            T qs = T(0);
            for (int sp = 0; sp < g.S; ++sp) qs += w[sp] * f.q_sun[sp * g.nd + u];
            sq_i += qi;
            sqc_i += qi * C;
            sq_s += qs;
            sqc_s += qs * C;
        }
    } else {
        int c = j - g.n_atm, y = c / g.nx, x = c - y * g.nx;
        for (int gd = 0; gd < g.ngd; ++gd) {
            int4 m = gp.gmem1[gd];
            T mun = f.mu_st[((m.z - 1) * g.ny + wrap_small(y + m.y, g.ny)) * g.nx + wrap_small(x + m.x, g.nx)];
            T C = dsqrt<T>(mus_lamb * mun) / (T)gp.gdist1[gd];
            T q = (T)gp.q_lamb[gd];
            sq_i += q;
            sqc_i += q * C;
        }
        sq_s = sq_i;
        sqc_s = sqc_i;
    }
    f.zc_iso[j] = (vc.coupling && sqc_i > T(0)) ? sq_i / sqc_i : T(0);
    f.zc_sun[j] = (vc.coupling && sqc_s > T(0)) ? sq_s / sqc_s : T(0);
}

// ---------------------------------------------------------------------------
// Fused edge march + edge weights: one warp per receiver row.  For every slot
// the optical depths of the chain segments come from the translation-
// invariant tap tables; the deposit fraction P, the quadrature weight q and
// the coupling c of the source give
//   K_ij = rho_i q_{j,u} c_{j,u} P          (stored, CSR order)
//   s_i  = sum_slots rho_i q^sun c^sun P e1_j
//   g_i  = sum_slots Theta_i(u . v) rho_i q^sun c^sun P e1_j   (atmospheric rows)

template <typename T>
__global__ void __launch_bounds__(256) k_assemble(GridC g, GraphP gp, FieldP<T> f, ViewC vc) {
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= g.n_nodes) return;
    const int e0 = gp.row_ptr[row], e1 = gp.row_ptr[row + 1];
    const T mus_lamb = (T)(vc.albedo * __longlong_as_double((long long)*f.mus_max_bits));
    const int ndir = g.nd + g.ngd;
    T rho, wr[MAX_SPECIES];
    if (row < g.n_atm) {
        T me = f.mu_e[row], ms = f.mu_st[row];
        rho = me > T(0) ? ms / me : T(0);
        for (int sp = 0; sp < g.S; ++sp)
            wr[sp] = ms > T(0) ? f.mu_s[(size_t)sp * g.n_atm + row] / ms : T(1) / (T)g.S;
    } else {
        rho = (T)vc.albedo;
        for (int sp = 0; sp < g.S; ++sp) wr[sp] = T(0);
    }
    T acc_s = T(0), acc_g = T(0);
    for (int e = e0 + lane; e < e1; e += 32) {
        const int j = gp.col[e];
        const DClass c = gp.cls[gp.code[e]];
        if (c.kind == 4) {  // padding
            f.val[e] = T(0);
            continue;
        }
        int bx, by, bz;
        if (j < g.n_atm) {
            bz = j / g.nxy;
            int r = j - bz * g.nxy;
            by = r / g.nx;
            bx = r - by * g.nx;
        } else {
            int r = j - g.n_atm;
            by = r / g.nx;
            bx = r - by * g.nx;
            bz = 0;
        }
        T tpre = c.pre_n ? tap_sum<T>(g, gp, f.mu_e, c.pre_off, c.pre_n, bx, by, bz) : T(0);
        T tseg = c.seg_n ? tap_sum<T>(g, gp, f.mu_e, c.seg_off, c.seg_n, bx, by, bz) : T(0);
        T thit = c.hit_n ? tap_sum<T>(g, gp, f.mu_e, c.hit_off, c.hit_n, bx, by, bz) : T(0);
        T P;
        if (c.kind == 0 || c.kind == 3) {  // chain node (atmospheric or ground source)
            T ep = dexp<T>(-tpre);
            if (c.bkind == 0) {
                P = ep * (-dexpm1<T>(-tseg));
            } else if (c.bkind == 1) {
                P = ep;
            } else {
                T tb = c.bkind == 2 ? f.tinf[(size_t)c.up_idx * g.n_atm + row]
                                    : (c.bkind == 3 ? thit : f.tinfg[(size_t)c.gdir * g.nxy + (j - g.n_atm)]);
                P = ep * (-dexpm1<T>(-(tseg + tb)));
            }
        } else if (c.kind == 1) {  // self deposit
            T tb = c.bkind == 2 ? f.tinf[(size_t)c.up_idx * g.n_atm + row] : thit;
            P = -dexpm1<T>(-tb);
        } else {  // ground hit
            P = (T)c.split * dexp<T>(-(tpre + thit));
        }
        T Wi, Ws;
        if (j < g.n_atm) {
            T mus = f.mu_st[j];
            T qi = (T)gp.q_iso[c.dir], qs = T(0);
            for (int sp = 0; sp < g.S; ++sp) {
                T w = mus > T(0) ? f.mu_s[(size_t)sp * g.n_atm + j] / mus : T(1) / (T)g.S;
                qs += w * f.q_sun[sp * g.nd + c.dir];
            }
            T ci = T(1), cs = T(1);
            if (!c.c_one) {
                T mun = c.n1_ground ? mus_lamb
                                    : f.mu_st[((bz + c.n1_dz) * g.ny + wrap_small(by + c.n1_dy, g.ny)) * g.nx +
                                              wrap_small(bx + c.n1_dx, g.nx)];
                T C = dsqrt<T>(mus * mun) * (T)c.dist1_inv;
                T zi = f.zc_iso[j], zs = f.zc_sun[j];
                ci = zi > T(0) ? C * zi : T(1);
                cs = zs > T(0) ? C * zs : T(1);
            }
            Wi = qi * ci;
            Ws = qs * cs;
        } else {
            T mun = f.mu_st[(c.n1_dz * g.ny + wrap_small(by + c.n1_dy, g.ny)) * g.nx + wrap_small(bx + c.n1_dx, g.nx)];
            T C = dsqrt<T>(mus_lamb * mun) * (T)c.dist1_inv;
            T z = f.zc_iso[j];
            T cc = z > T(0) ? C * z : T(1);
            Wi = (T)gp.q_lamb[c.gdir] * cc;
            Ws = Wi;
        }
        f.val[e] = rho * Wi * P;
        T sun = rho * Ws * P * f.e1[j];
        acc_s += sun;
        T th = T(0);
        for (int sp = 0; sp < g.S; ++sp) th += wr[sp] * f.hgv[sp * ndir + c.hgdir];
        acc_g += th * sun;
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc_s += __shfl_xor_sync(0xffffffffu, acc_s, o);
        acc_g += __shfl_xor_sync(0xffffffffu, acc_g, o);
    }
    if (lane == 0) {
        f.s[row] = acc_s;
        if (row < g.n_atm) f.gsun[row] = acc_g;
    }
}

template <typename T>
void launch_assemble_pre(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                         const ViewP &vp, long long *launches) {
    const int th = 256;
    cudaMemsetAsync(f.mus_max_bits, 0, sizeof(unsigned long long), st);
    k_prep<T><<<(g.n_atm + th - 1) / th, th, 0, st>>>(g, f);
    k_tables<T><<<g.S, 256, sizeof(double) * g.nd, st>>>(g, f, vc, vp);
    k_sun<T><<<(g.n_nodes + th - 1) / th, th, 0, st>>>(g, f, vc, vp);
    long long nt = (long long)g.nup * g.R * g.nxy;
    k_tinf<T><<<(unsigned)((nt + th - 1) / th), th, 0, st>>>(g, gp, f);
    k_tinfg<T><<<(g.ngd * g.nxy + th - 1) / th, th, 0, st>>>(g, gp, f);
    k_znorm<T><<<(g.n_nodes + th - 1) / th, th, 0, st>>>(g, gp, f, vc);
    if (launches) *launches += 6;
}

template <typename T>
void launch_assemble_rows(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                          long long *launches) {
    const int th = 256;
    long long nthr = (long long)g.n_nodes * 32;
    k_assemble<T><<<(unsigned)((nthr + th - 1) / th), th, 0, st>>>(g, gp, f, vc);
    if (launches) *launches += 1;
}

#define INST(T)                                                                                                   \
    template void launch_assemble_pre<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,          \
                                         const ViewC &, const ViewP &, long long *);                              \
    template void launch_assemble_rows<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,         \
                                          const ViewC &, long long *);
INST(float)
INST(double)
#undef INST

}  // namespace tk
