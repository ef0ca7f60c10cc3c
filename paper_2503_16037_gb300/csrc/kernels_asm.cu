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
        {
            T *mx = f.mu_x + (size_t)z * 4 * g.nxy + (size_t)y * 2 * g.nx + x;
            mx[0] = a + s;
            mx[g.nx] = a + s;
            mx[(size_t)g.ny * 2 * g.nx] = a + s;
            mx[(size_t)g.ny * 2 * g.nx + g.nx] = a + s;
        }
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
    if (threadIdx.x < 32) {  // one warp: strided partial sums, then a fixed butterfly
        double t = 0.0;
        for (int u = threadIdx.x; u < g.nd; u += 32) t += f.cellsum[sp * g.nd + u];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) total = t;
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

// Long rays (the direct beam here, the ground chains' rays to the TOA in
// k_tinfg): every ray of a block shares one tap list (the block's rows lie in
// one layer), which is staged in shared memory in chunks of kRayChunk taps,
// each tap as one offset into the extinction repeated 2 x 2 horizontally
// (a tap's column offsets are stored wrapped into [0, nx) x [0, ny), so the
// base column plus the offset never wraps twice); each thread sums its own
// ray in four interleaved partial sums (taps t = s mod 4), combined as
// (a0 + a1) + (a2 + a3), so the extinction gathers of a warp are coalesced
// along x and four are in flight per thread.
constexpr int kRayChunk = 512;
constexpr int kRayBlock = 128;

template <typename T>
struct RayTap {
    int off;  // cell offset in the extended extinction (FieldP::mu_x) from the ray's base column
    T len;
};

template <typename T>
__device__ __forceinline__ T ray_tau_block(const GridC &g, const RTap *__restrict__ taps, const T *__restrict__ len,
                                           const T *__restrict__ mu_x, int off, int n, int x, int y,
                                           RayTap<T> *stap) {
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    const T *base = mu_x + y * 2 * g.nx + x;
    auto tap = [&](int t) -> T {
        const RayTap<T> r = stap[t];
        return r.len * __ldg(base + r.off);
    };
    for (int c0 = 0; c0 < n; c0 += kRayChunk) {
        const int cn = min(kRayChunk, n - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cn; t += blockDim.x) {
            const int2 r = __ldg(reinterpret_cast<const int2 *>(taps + off + c0 + t));
            // r.y = dz nx ny: the layer's offset in mu_x is 4 r.y
            RayTap<T> e;
            e.off = 4 * r.y + (r.x >> 16) * 2 * g.nx + (r.x & 0xffff);
            e.len = __ldg(len + off + c0 + t);
            stap[t] = e;
        }
        __syncthreads();
        int t = 0;
        for (; t + 4 <= cn; t += 4) {
            a0 += tap(t);
            a1 += tap(t + 1);
            a2 += tap(t + 2);
            a3 += tap(t + 3);
        }
        if (t < cn) a0 += tap(t);
        if (t + 1 < cn) a1 += tap(t + 1);
        if (t + 2 < cn) a2 += tap(t + 2);
    }
    return (a0 + a1) + (a2 + a3);
}

// The direct beam of node (x, y) of layer L (nz: the ground), r its index in
// the layer (r >= nxy: a padding thread, which still takes part in the
// block's tap staging): T_sun from the ray's optical depth, e1, and their
// stores; returns e1 (0 for padding threads).
template <typename T>
__device__ __forceinline__ T sun_node(const GridC &g, const FieldP<T> &f, const ViewC &vc, const ViewP &vp, int L,
                                      int r, int x, int y, RayTap<T> *stap) {
    const int Zs = L < g.nz ? L + 1 : 0;  // ray start: top face of layer L, or the ground point
    const T *len;
    if constexpr (sizeof(T) == 4)
        len = (const T *)vp.sun_len_f;
    else
        len = (const T *)vp.sun_len_d;
    const T tau = ray_tau_block<T>(g, vp.sun_rt, len, f.mu_x, __ldg(vp.sun_off + Zs), __ldg(vp.sun_n + Zs), x, y,
                                   stap);
    if (r >= g.nxy) return T(0);
    const T Ts = dexp<T>(-tau);
    const T base = (T)(vc.f0 * vc.mu0 * g.hx * g.hy);
    if (L < g.nz) {
        const int i = L * g.nxy + r;
        f.tsun[i] = Ts;
        const T me = f.mu_e[i];
        const T om = me > T(0) ? f.mu_st[i] / me : T(0);
        const T e = om * base * Ts * (-dexpm1<T>(-me * (T)(g.hz / vc.mu0)));
        f.e1[i] = e;
        store_halo(f.e1_h, g, x, y, L, e);
        return e;
    }
    const int i = g.n_atm + r;
    f.tsun[i] = Ts;
    const T e = (T)vc.albedo * base * Ts;
    f.e1[i] = e;
    store_halo(f.e1_h, g, x, y, g.nz, e);
    return e;
}

// grid (ceil(nxy / kRayBlock), nz + 1): blockIdx.y = node layer (nz: the ground)
template <typename T>
__global__ void __launch_bounds__(kRayBlock) k_sun(GridC g, FieldP<T> f, ViewC vc, ViewP vp) {
    __shared__ RayTap<T> stap[kRayChunk];
    const int r = blockIdx.x * kRayBlock + threadIdx.x;
    const int rr = r < g.nxy ? r : 0;
    const int y = rr / g.nx, x = rr - y * g.nx;
    sun_node<T>(g, f, vc, vp, blockIdx.y, r, x, y, stap);
}

// ---------------------------------------------------------------------------
// Optical depth of the lattice segment from every voxel centre a to a + u, for
// each canonical direction u (one of each pair {u, -u}); a segment traversed
// backwards (-u, from a + u) reads the same entry.  A block of kSegTX x kSegTY
// voxels of one layer copies the extinction it reaches (its columns and rows
// +- H, its layer and the R above: every tap of a canonical segment lies
// there, checked on the host) into shared memory, with the taps of all
// canonical segments as offsets into that tile; entries whose end lies above
// the TOA are not used and are set to 0.
constexpr int kSegHmax = 2;
constexpr int kSegTile = (kSegHmax + 1) * (kSegTY + 2 * kSegHmax) * (kSegTX + 2 * kSegHmax);

template <typename T>
__global__ void __launch_bounds__(kSegTX * kSegTY) k_segtau(GridC g, GraphP gp, FieldP<T> f) {
    __shared__ T tile[kSegTile];
    __shared__ int toff[kSegMaxTaps];
    __shared__ T tlen[kSegMaxTaps];
    __shared__ int4 cs[64];
    const int H = g.H, TXh = kSegTX + 2 * H, TYh = kSegTY + 2 * H, tpl = TXh * TYh;
    const int x0 = blockIdx.x * kSegTX, y0 = blockIdx.y * kSegTY, z = blockIdx.z;
    const T *len = tap_len<T>(gp);
    for (int c = threadIdx.x; c < g.nc; c += blockDim.x) cs[c] = __ldg(gp.cseg + c);
    for (int t = threadIdx.x; t < gp.nctap; t += blockDim.x) {
        const int gi = __ldg(gp.ctap + t);
        const DTap d = gp.taps[gi];
        toff[t] = d.dz * tpl + d.dy * TXh + d.dx;
        tlen[t] = __ldg(len + gi);
    }
    for (int e = threadIdx.x; e < (g.R + 1) * tpl; e += blockDim.x) {
        const int tz = e / tpl, rem = e - tz * tpl, tr = rem / TXh, tc = rem - tr * TXh;
        T v = T(0);
        if (z + tz < g.nz && x0 + tc < g.nxp && y0 + tr < g.nyp)
            v = __ldg(f.mu_e_h + (size_t)(z + tz) * g.lp + (size_t)(y0 + tr) * g.nxp + x0 + tc);
        tile[e] = v;
    }
    __syncthreads();
    const int tx = threadIdx.x % kSegTX, ty = threadIdx.x / kSegTX;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= g.nx || y >= g.ny) return;
    const int p = (int)halo_pos(g, x, y, z);
    const int ax = x < H ? g.nx : (x >= g.nx - H ? -g.nx : 0);
    const int ay = y < H ? g.ny * g.nxp : (y >= g.ny - H ? -g.ny * g.nxp : 0);
    const T *tb = tile + (ty + H) * TXh + tx + H;
    for (int c = 0; c < g.nc; ++c) {
        const int4 sc = cs[c];
        T tau = T(0);
        if (z + sc.z < g.nz)
            for (int k = sc.x; k < sc.x + sc.y; ++k) tau += tlen[k] * tb[toff[k]];
        T *o = f.tseg + (size_t)c * g.npad + p;
        o[0] = tau;
        if (ax) o[ax] = tau;
        if (ay) {
            o[ay] = tau;
            if (ax) o[ax + ay] = tau;
        }
    }
}


// The same table with the canonical segments as kernel parameters (SegTab):
// the direction and tap loops have fixed trip counts, so every tile offset and
// length is a parameter operand and nothing but the tile reads and the
// multiply-adds remain per tap (zero-length padding taps included).
template <typename T, int R, int NC>
__global__ void __launch_bounds__(kSegTX * kSegTY) k_segtau_fixed(GridC g, FieldP<T> f,
                                                                 const __grid_constant__ SegTab<T> tab) {
    constexpr int H = R, TXh = kSegTX + 2 * H, TYh = kSegTY + 2 * H, tpl = TXh * TYh;
    __shared__ T tile[(R + 1) * tpl];
    const int x0 = blockIdx.x * kSegTX, y0 = blockIdx.y * kSegTY, z = blockIdx.z;
    for (int e = threadIdx.x; e < (R + 1) * tpl; e += kSegTX * kSegTY) {
        const int tz = e / tpl, rem = e - tz * tpl, tr = rem / TXh, tc = rem - tr * TXh;
        T v = T(0);
        if (z + tz < g.nz && x0 + tc < g.nxp && y0 + tr < g.nyp)
            v = __ldg(f.mu_e_h + (size_t)(z + tz) * g.lp + (size_t)(y0 + tr) * g.nxp + x0 + tc);
        tile[e] = v;
    }
    __syncthreads();
    const int tx = threadIdx.x % kSegTX, ty = threadIdx.x / kSegTX;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= g.nx || y >= g.ny) return;
    const int p = (int)halo_pos(g, x, y, z);
    const int ax = x < H ? g.nx : (x >= g.nx - H ? -g.nx : 0);
    const int ay = y < H ? g.ny * g.nxp : (y >= g.ny - H ? -g.ny * g.nxp : 0);
    const T *tb = tile + (ty + H) * TXh + tx + H;
    T *o = f.tseg + p;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        T tau = T(0);
        if (z + tab.uz[c] < g.nz) {
#pragma unroll
            for (int k = 0; k < kSegTapsPer; ++k) tau += tab.len[c][k] * tb[tab.off[c][k]];
        }
        o[0] = tau;
        if (ax) o[ax] = tau;
        if (ay) {
            o[ay] = tau;
            if (ax) o[ax + ay] = tau;
        }
        o += g.npad;
    }
}

// Optical depth from each voxel centre to the TOA along each upward lattice
// direction, by recursion down the lattice lines:
//   tau_inf(j, u) = tau(j -> j + u) + tau_inf(j + u, u).
// One thread per (upward direction, start layer offset, column).  The
// segment depths of kTinfBatch steps are loaded before they are added, so the
// loads of a batch are in flight together; the sum runs in the same order as
// a plain walk.
constexpr int kTinfBatch = 8;

template <typename T>
__global__ void k_tinf(GridC g, GraphP gp, FieldP<T> f) {
    const int ui = blockIdx.y, rem = blockIdx.x * blockDim.x + threadIdx.x;
    if (rem >= g.R * g.nxy) return;
    const int o = rem / g.nxy, c = rem - o * g.nxy;
    const int u = __ldg(gp.up_dirs + ui);
    const int4 d = gp.dirs[u];
    if (o >= d.z) return;
    const int zt = g.nz - 1 - o;
    if (zt < 0) return;
    int y = c / g.nx, x = c - y * g.nx;
    T tau = tap_sum<T>(g, gp, f.mu_e, gp.top_off[ui * g.R + o], gp.top_n[ui * g.R + o], x, y, zt);
    T *out = f.tinf + (size_t)ui * g.n_atm;
    out[(zt * g.ny + y) * g.nx + x] = tau;
    const T *seg = f.tseg + (size_t)__ldg(gp.up_canon + ui) * g.npad;
    for (int z0 = zt - d.z; z0 >= 0; z0 -= kTinfBatch * d.z) {
        int idx[kTinfBatch];
        T v[kTinfBatch];
#pragma unroll
        for (int b = 0; b < kTinfBatch; ++b) {
            const int z = z0 - b * d.z;
            x = wrap_small(x - d.x, g.nx);
            y = wrap_small(y - d.y, g.ny);
            idx[b] = (z * g.ny + y) * g.nx + x;
            v[b] = z >= 0 ? __ldg(seg + halo_pos(g, x, y, z)) : T(0);
        }
#pragma unroll
        for (int b = 0; b < kTinfBatch; ++b) {
            if (z0 - b * d.z >= 0) {
                tau += v[b];
                out[idx[b]] = tau;
            }
        }
    }
}

// ground chains: optical depth from the terminal member to the TOA, one
// thread per (ground direction, column); grid (ceil(nxy / kRayBlock), ngd)
template <typename T>
__global__ void __launch_bounds__(kRayBlock) k_tinfg(GridC g, GraphP gp, FieldP<T> f) {
    __shared__ RayTap<T> stap[kRayChunk];
    const int gd = blockIdx.y;
    const int r = blockIdx.x * kRayBlock + threadIdx.x;
    const int rr = r < g.nxy ? r : 0;
    const int y = rr / g.nx, x = rr - y * g.nx;
    const T tau = ray_tau_block<T>(g, gp.rtaps, tap_len<T>(gp), f.mu_x, __ldg(gp.gtop_off + gd),
                                   __ldg(gp.gtop_n + gd), x, y, stap);
    // haloed plane of ground direction gd: layer index 0 of a (1 x lp) array
    if (r < g.nxy) store_halo(f.tinfg + (size_t)gd * g.lp, g, x, y, 0, tau);
}

// ---------------------------------------------------------------------------
// Coupling normalisers (Eq. scatt_coup as a routing weight): for each source
//   zc = sum_{U_c} q / sum_{U_c} q C   (0 when the coupling is off or the
// denominator vanishes), so that c_{j,u} = C_{j,u} zc and sum_u q c = 1,
// with C_{j,u} = sqrt(mu_s(j)) sqrt(mu_s(n1)) / d.  U_c: directions whose
// chain has a receiver other than the source.  Which directions have a
// receiver depends on the source's layer only, so a block of one layer lists
// them once in shared memory, each with its weights q / d (iso and, per
// species, sun), and a thread sums them over sqrt(mu_s) of its source's first
// receivers (a stencil sum over the haloed sqrt(mu_s)); ground receivers add
// a per-layer constant.  The stored factors are premultiplied by sqrt(mu_s)
// of the source: c = a sqrt(mu_s(n1)) / d.  The same pass writes the edge
// kernel's source records (FieldP::srec), whose sun factors need e1, so it
// first traces the direct beam of its nodes (k_sunz).
constexpr int kZnBlock = 128;
constexpr int kZnMaxDir = 128;

template <typename T, int S>
__global__ void __launch_bounds__(kZnBlock) k_sunz(GridC g, GraphP gp, FieldP<T> f, ViewC vc, ViewP vp) {
    __shared__ RayTap<T> stap[kRayChunk];
    __shared__ int sdh[kZnMaxDir];
    __shared__ T sw[kZnMaxDir][1 + S];
    __shared__ T sq[kZnMaxDir][1 + S];   // q of the directions with a receiver (0: none)
    __shared__ T sg[kZnMaxDir][1 + S];   // ground-receiver part of q C / (sqrt(mu_s(j)) sqrt(mu_s^Lamb))
    __shared__ T cst[2][1 + S];          // per layer: sum q, ground constant
    const int L = blockIdx.y;
    const bool ground = L == g.nz;
    const int ndir = ground ? g.ngd : g.nd;
    // the direct beam of the block's nodes (the rays of k_sun), kept for the
    // source records below
    T e1;
    {
        const int r = blockIdx.x * kZnBlock + threadIdx.x;
        const int rr = r < g.nxy ? r : 0;
        const int y = rr / g.nx, x = rr - y * g.nx;
        e1 = sun_node<T>(g, f, vc, vp, L, r, x, y, stap);
    }
    const T rt_lamb = dsqrt<T>((T)(vc.albedo * __longlong_as_double((long long)*f.mus_max_bits)));
    for (int u = threadIdx.x; u < ndir; u += blockDim.x) {
        T w[1 + S], qq[1 + S], gg[1 + S];
        int dh = 0;
        if (!ground) {
            const int4 d = gp.dirs[u];
            const int rz = L + d.z;
            const T qi = Cst<T>::q_iso(gp, u), il = T(1) / Cst<T>::dir_len(gp, u);
            T qs[S];
#pragma unroll
            for (int sp = 0; sp < S; ++sp) qs[sp] = f.q_sun[sp * g.nd + u];
            const bool atm = rz >= 0 && rz < g.nz, gnd = rz < 0;
            dh = atm ? __ldg(gp.dir_h + u) : 0;
            // ground receiver: d = (z + 1/2) / (-u_z) |u|, sqrt(mu_s) of the surface rt_lamb
            const T gf = gnd ? rt_lamb * (T)(-d.z) / ((T)L + T(0.5)) : T(0);
            w[0] = atm ? qi * il : T(0);
            qq[0] = (atm || gnd) ? qi : T(0);
            gg[0] = qi * il * gf;
#pragma unroll
            for (int sp = 0; sp < S; ++sp) {
                w[1 + sp] = atm ? qs[sp] * il : T(0);
                qq[1 + sp] = (atm || gnd) ? qs[sp] : T(0);
                gg[1 + sp] = qs[sp] * il * gf;
            }
        } else {
            const int4 m = gp.gmem1[u];
            // first member (x + m.x, y + m.y, layer m.z - 1) from the ground node's haloed position
            dh = (m.z - 1 - g.nz) * g.lp + m.y * g.nxp + m.x;
            const T q = Cst<T>::q_lamb(gp, u), il = T(1) / Cst<T>::gdist1(gp, u);
#pragma unroll
            for (int k = 0; k <= S; ++k) {
                w[k] = q * il;
                qq[k] = q;
                gg[k] = T(0);
            }
        }
        sdh[u] = dh;
#pragma unroll
        for (int k = 0; k <= S; ++k) {
            sw[u][k] = w[k];
            sq[u][k] = qq[k];
            sg[u][k] = gg[k];
        }
    }
    __syncthreads();
    if (threadIdx.x <= S) {  // fixed-order sums of the per-layer constants
        const int k = threadIdx.x;
        T a = T(0), b = T(0);
        for (int u = 0; u < ndir; ++u) {
            a += sq[u][k];
            b += sg[u][k];
        }
        cst[0][k] = a;
        cst[1][k] = b;
    }
    __syncthreads();
    const int r = blockIdx.x * kZnBlock + threadIdx.x;
    if (r >= g.nxy) return;
    const int y = r / g.nx, x = r - y * g.nx;
    const int p = (int)halo_pos(g, x, y, L);
    T acc[1 + S];
#pragma unroll
    for (int k = 0; k <= S; ++k) acc[k] = cst[1][k];
    const T *rth = f.rt_h + p;
#pragma unroll 4
    for (int u = 0; u < ndir; ++u) {
        const T rtn = __ldg(rth + sdh[u]);
#pragma unroll
        for (int k = 0; k <= S; ++k) acc[k] += sw[u][k] * rtn;
    }
    const int i = ground ? g.n_atm + r : L * g.nxy + r;
    T rt_src, sq_i = cst[0][0], sq_s, sqc_i, sqc_s;
    T wv[S];
    if (!ground) {
        rt_src = f.rt[i];
        sq_s = T(0);
        T cs = T(0);
#pragma unroll
        for (int sp = 0; sp < S; ++sp) {
            wv[sp] = f.wsp[(size_t)sp * g.n_atm + i];
            sq_s += wv[sp] * cst[0][1 + sp];
            cs += wv[sp] * acc[1 + sp];
        }
        sqc_i = rt_src * acc[0];
        sqc_s = rt_src * cs;
    } else {
        rt_src = rt_lamb;
        sqc_i = rt_src * acc[0];
        sq_s = sq_i;
        sqc_s = sqc_i;
    }
    const T ai = (vc.coupling && sqc_i > T(0)) ? sq_i / sqc_i * rt_src : T(0);
    const T as = (vc.coupling && sqc_s > T(0)) ? sq_s / sqc_s * rt_src : T(0);
    store_halo(f.a_iso, g, x, y, L, ai);
    store_halo(f.a_sun, g, x, y, L, as);
    // the edge kernel's source record: a_iso, then per species wsp e1 a_sun
    // (negated when c^sun = 1; a ground source: e1 a_iso, negated when c = 1)
    constexpr int RS = srec_stride(S);
    T rec[RS];
    rec[0] = ai;
#pragma unroll
    for (int k = 1; k < RS; ++k) {
        const int sp = k - 1;
        if (sp >= S)
            rec[k] = T(0);
        else if (!ground)
            rec[k] = wv[sp < S ? sp : 0] * e1 * (as > T(0) ? as : T(-1));
        else
            rec[k] = sp == 0 ? e1 * (ai > T(0) ? ai : T(-1)) : T(0);
    }
    const long long pp = halo_pos(g, x, y, L);
    const int axo = x < g.H ? g.nx : (x >= g.nx - g.H ? -g.nx : 0);
    const int ayo = y < g.H ? g.ny * g.nxp : (y >= g.ny - g.H ? -g.ny * g.nxp : 0);
    const long long cp[4] = {pp, pp + axo, pp + ayo, pp + axo + ayo};
    const bool cw[4] = {true, axo != 0, ayo != 0, axo != 0 && ayo != 0};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (!cw[q]) continue;
        T *o = f.srec + cp[q] * RS;
#pragma unroll
        for (int k = 0; k < RS; ++k) o[k] = rec[k];
    }
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

// The edge kernel of the default assembly (full stencil, node unknowns): the
// same rows, slots and values as k_asm in mode 0 with fewer lookups per
// slot.  Per source it reads one record (FieldP::srec: a_iso and the sun
// factors g_sp = w_sp e1 a_sun, negated when the source's sun weight is 1),
// so that
//   W_iso       = q c^iso = a_iso sqrt(mu_s(n1)) q / d   (q when a_iso = 0)
//   W_sun e1    = sum_sp g_sp q^sun_sp (sqrt(mu_s(n1)) / d, or -1 when negated);
// sqrt(mu_s(n1)) is the row's own value when the first receiver is the
// receiver itself (bit 12 of the descriptor); only the optical depths the
// slot's kind needs are read.  g^sun is accumulated per species (the species
// weights of the receiver applied once at the end).  The block first copies
// its layer's template (the slot descriptors, with each slot's q^sun and HG
// weight toward the instrument per species looked up once) into shared
// memory, so a warp's step to its next slot costs a shared-memory read
// instead of a dependent global round trip.
template <typename T, int RS>
struct Rec;
template <>
struct Rec<float, 4> {
    __device__ static __forceinline__ void load(const float *p, float *v) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
        v[3] = a.w;
    }
};
template <>
struct Rec<float, 8> {
    __device__ static __forceinline__ void load(const float *p, float *v) {
        Rec<float, 4>::load(p, v);
        Rec<float, 4>::load(p + 4, v + 4);
    }
};
template <int RS>
struct Rec<double, RS> {
    __device__ static __forceinline__ void load(const double *p, double *v) {
#pragma unroll
        for (int k = 0; k < RS; k += 2) {
            const double2 a = __ldg(reinterpret_cast<const double2 *>(p + k));
            v[k] = a.x;
            v[k + 1] = a.y;
        }
    }
};

// 1 - exp(-t) for t >= 0 without branches: t (1 - t/2 + t^2/6 - t^3/24 +
// t^4/120) below t = 1/8 (truncation below 5e-8 relative), 1 - exp(-t) above
// (cancellation there is at most a factor 8.5); FP64: expm1.
template <typename T>
__device__ __forceinline__ T q_of(T t);
template <>
__device__ __forceinline__ float q_of<float>(float t) {
    const float e = __expf(-t);
    const float p = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.f / 120.f, -1.f / 24.f), 1.f / 6.f), -0.5f), 1.f);
    return t < 0.125f ? p : 1.f - e;
}
template <>
__device__ __forceinline__ double q_of<double>(double t) { return -expm1(-t); }

// The common slot kinds of an atmospheric source (descriptor bits 13-14,
// assigned on the host), each with straight-line code over the lane's four
// rows: 1 a chain node before the end of its chain, P = T_pre Q(tau_seg);
// 2 the terminal node with nothing beyond, P = T_pre; 3 the terminal node of
// an upward chain, P = T_pre Q(tau_seg + tau_inf).  PRE: the chain has
// segments before the receiver (then the first receiver is not the
// receiver itself).  T = exp(-tau), Q = 1 - T.
template <typename T, int S, int FT, bool PRE>
__device__ __forceinline__ void slot_fast(const GridC &g, const FieldP<T> &f, const GroupRows &G, const int (&rowc)[4],
                                          const T (&rho)[4], const T (&rtr)[4], int src, int pre, int seg, int n1,
                                          int aux, T q, T qd, T dinv, const T (&qsun)[S], const T (&hv)[S],
                                          T (&kv)[4], T (&acc_s)[4], T (&acc_g)[4][S]) {
    constexpr int RS = srec_stride(S);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int rp = G.rp[k], j = rp + src;
        T ep = T(1);
        if (PRE) ep = fast_exp_neg<T>(__ldg(f.tseg + pre + rp));
        T P;
        if (FT == 2) {
            P = ep;
        } else {
            T ts = __ldg(f.tseg + seg + rp);
            if (FT == 3) ts += __ldg(f.tinf + (size_t)aux * g.n_atm + rowc[k]);
            P = ep * q_of<T>(ts);
        }
        const T rtn = PRE ? __ldg(f.rt_h + rp + n1) : rtr[k];
        T rec[RS];
        Rec<T, RS>::load(f.srec + (size_t)j * RS, rec);
        const T Wi = rec[0] > T(0) ? rec[0] * (rtn * qd) : q;
        T m = T(0);
#pragma unroll
        for (int sp = 0; sp < S; ++sp) m += rec[1 + sp] * qsun[sp];
        const T se = m < T(0) ? -m : m * (rtn * dinv);
        const T rP = rho[k] * P;
        kv[k] = rP * Wi;
        const T sun = rP * se;
        acc_s[k] += sun;
#pragma unroll
        for (int sp = 0; sp < S; ++sp) acc_g[k][sp] += hv[sp] * sun;
    }
}

// Warps per group and register budget (blocks per SM) of k_asm0.
#ifndef TK_ASM0_W
#define TK_ASM0_W 8
#endif
#ifndef TK_ASM0_MINB
#define TK_ASM0_MINB 3
#endif
// dynamic shared memory of k_asm0: the staged template (stage_template);
// after the slot loop the same space holds the warps' partial sums of s and
// g^sun ([W][4 + 4 S][32])
template <typename T, int W>
inline size_t asm0_smem(const GridC &g) {
    const size_t desc = template_smem<T>(g);
    const size_t red = (size_t)W * (4 + 4 * g.S) * 32 * sizeof(T);
    return desc > red ? desc : red;
}
template <typename T, int S, int W, int MINB>
__global__ void __launch_bounds__(32 * W, MINB)
    k_asm0(GridC g, GraphP gp, FieldP<T> f, ViewC vc) {
    constexpr int RS = srec_stride(S);
    constexpr int NW = aslot_words<T>();
    extern __shared__ __align__(16) unsigned char asm0_dyn[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const GroupRows G = group_rows(g, gp, blockIdx.x);
    const bool ground_row = G.z == g.nz;
    int4 *sdesc = reinterpret_cast<int4 *>(asm0_dyn);
    T *sconst = reinterpret_cast<T *>(sdesc + (size_t)NW * G.nt);
    // the group's template: descriptors and the per-slot direction constants
    stage_template<T, S>(g, gp, f, G.t0, G.nt, ground_row, sdesc, sconst);
    __syncthreads();
    const T rt_lamb = dsqrt<T>((T)(vc.albedo * __longlong_as_double((long long)*f.mus_max_bits)));
    T rho[4], rtr[4];
    int rowc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        rowc[k] = G.row[k] >= 0 ? G.row[k] : G.z * g.nxy;  // rows past the layer's end read a valid node
        rtr[k] = __ldg(f.rt_h + G.rp[k]);
        if (!ground_row) {
            const T me = f.mu_e[rowc[k]], ms = f.mu_st[rowc[k]];
            rho[k] = me > T(0) ? ms / me : T(0);
        } else {
            rho[k] = (T)vc.albedo;
        }
    }
    T acc_s[4] = {T(0), T(0), T(0), T(0)}, acc_g[4][S];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int sp = 0; sp < S; ++sp) acc_g[k][sp] = T(0);
    T *vout = f.val + G.vb + 4 * lane;
    for (int t = w; t < G.nt; t += W) {
        int4 a0, a1, a2;
        int hit_off;
        T q, dinv, split;
        T qsun[S], hv[S];
        {
            const StagedSlot<T> d = staged_slot<T>(sdesc, t);
            a0 = d.a0;
            a1 = d.a1;
            a2 = d.a2;
            hit_off = d.hit_off;
            q = d.q;
            dinv = d.dinv;
            split = d.split;
#pragma unroll
            for (int sp = 0; sp < S; ++sp) {
                qsun[sp] = sconst[(size_t)t * 2 * S + sp];
                hv[sp] = sconst[(size_t)t * 2 * S + S + sp];
            }
        }
        const int src = a0.x, pre = a0.y, seg = a0.z, n1 = a0.w;
        const int aux = a1.x, tbase = a1.y, bits = a1.z;
        const int taps = a2.y, pre_off = a2.z, seg_off = a2.w;
        const int kind = bits & 15, bkind = (bits >> 4) & 15;
        const bool c_one = (bits >> 8) & 1, n1_ground = (bits >> 9) & 1, has_pre = (bits >> 10) & 1;
        const bool n1_row = (bits >> 12) & 1;
        const int ft = (bits >> 13) & 3;
        const int pre_n = taps & 0xff, seg_n = (taps >> 8) & 0xff, hit_n = (taps >> 16) & 0xff;
        const T qd = q * dinv;
        T kv[4];
        if (ft == 1) {
            if (has_pre)
                slot_fast<T, S, 1, true>(g, f, G, rowc, rho, rtr, src, pre, seg, n1, aux, q, qd, dinv, qsun, hv, kv,
                                         acc_s, acc_g);
            else
                slot_fast<T, S, 1, false>(g, f, G, rowc, rho, rtr, src, pre, seg, n1, aux, q, qd, dinv, qsun, hv, kv,
                                          acc_s, acc_g);
        } else if (ft == 2) {
            if (has_pre)
                slot_fast<T, S, 2, true>(g, f, G, rowc, rho, rtr, src, pre, seg, n1, aux, q, qd, dinv, qsun, hv, kv,
                                         acc_s, acc_g);
            else
                slot_fast<T, S, 2, false>(g, f, G, rowc, rho, rtr, src, pre, seg, n1, aux, q, qd, dinv, qsun, hv, kv,
                                          acc_s, acc_g);
        } else if (ft == 3) {
            if (has_pre)
                slot_fast<T, S, 3, true>(g, f, G, rowc, rho, rtr, src, pre, seg, n1, aux, q, qd, dinv, qsun, hv, kv,
                                         acc_s, acc_g);
            else
                slot_fast<T, S, 3, false>(g, f, G, rowc, rho, rtr, src, pre, seg, n1, aux, q, qd, dinv, qsun, hv, kv,
                                          acc_s, acc_g);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int rp = G.rp[k];
                const int j = rp + src;
                // deposit fraction P of the slot (chain lumping of what lies beyond)
                T P;
                if (kind == 0 || kind == 3) {  // chain node (atmospheric or ground source)
                    T ep = T(1);
                    if (has_pre) {
                        const T tpre = pre >= 0 ? __ldg(f.tseg + pre + rp)
                                                : tap_sum_h<T>(gp, f.mu_e_h, pre_off, pre_n, rp + tbase);
                        ep = fast_exp_neg<T>(tpre);
                    }
                    if (bkind == 1) {
                        P = ep;
                    } else {
                        T ts = seg >= 0 ? __ldg(f.tseg + seg + rp)
                                        : (seg_n ? tap_sum_h<T>(gp, f.mu_e_h, seg_off, seg_n, rp + tbase) : T(0));
                        if (bkind == 2)
                            ts += __ldg(f.tinf + (size_t)aux * g.n_atm + rowc[k]);
                        else if (bkind == 3)
                            ts += tap_sum_h<T>(gp, f.mu_e_h, hit_off, hit_n, rp + tbase);
                        else if (bkind == 4)
                            ts += __ldg(f.tinfg + aux + rp);
                        P = ep * q_of<T>(ts);
                    }
                } else if (kind == 1) {  // self deposit
                    const T tb = bkind == 2 ? __ldg(f.tinf + (size_t)aux * g.n_atm + rowc[k])
                                            : tap_sum_h<T>(gp, f.mu_e_h, hit_off, hit_n, rp + tbase);
                    P = q_of<T>(tb);
                } else {  // ground hit
                    const T tpre = pre >= 0 ? __ldg(f.tseg + pre + rp)
                                            : (pre_n ? tap_sum_h<T>(gp, f.mu_e_h, pre_off, pre_n, rp + tbase) : T(0));
                    const T thit = tap_sum_h<T>(gp, f.mu_e_h, hit_off, hit_n, rp + tbase);
                    P = split * fast_exp_neg<T>(tpre + thit);
                }
                // weights: W_iso and W_sun e1 of the source's chain
                T Wi, se;
                if (c_one) {  // no receiver other than the source: c = 1
                    T m = T(0);
#pragma unroll
                    for (int sp = 0; sp < S; ++sp) m += __ldg(f.wsp_h + (size_t)sp * g.npad + j) * qsun[sp];
                    Wi = q;
                    se = m * __ldg(f.e1_h + j);
                } else {
                    const T rtn = n1_row ? rtr[k] : (n1_ground ? rt_lamb : __ldg(f.rt_h + rp + n1));
                    T rec[RS];
                    Rec<T, RS>::load(f.srec + (size_t)j * RS, rec);
                    Wi = rec[0] > T(0) ? rec[0] * (rtn * qd) : q;
                    T m = T(0);
#pragma unroll
                    for (int sp = 0; sp < S; ++sp) m += rec[1 + sp] * qsun[sp];
                    se = m < T(0) ? -m : m * (rtn * dinv);
                }
                const T rP = rho[k] * P;
                kv[k] = rP * Wi;
                const T sun = rP * se;
                acc_s[k] += sun;
#pragma unroll
                for (int sp = 0; sp < S; ++sp) acc_g[k][sp] += hv[sp] * sun;
            }
        }
        st_quad_cs(vout + (size_t)t * kGroup, kv);
    }
    __syncthreads();  // every warp is done with the staged template
    T(*sh)[4 + 4 * S][32] = reinterpret_cast<T(*)[4 + 4 * S][32]>(asm0_dyn);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        sh[w][k][lane] = acc_s[k];
#pragma unroll
        for (int sp = 0; sp < S; ++sp) sh[w][4 + 4 * sp + k][lane] = acc_g[k][sp];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (G.row[k] < 0) continue;
            T a = T(0);
#pragma unroll
            for (int qq = 0; qq < W; ++qq) a += sh[qq][k][lane];
            f.s[G.row[k]] = a;
            if (!ground_row) {
                T b = T(0);
#pragma unroll
                for (int sp = 0; sp < S; ++sp) {
                    T c = T(0);
#pragma unroll
                    for (int qq = 0; qq < W; ++qq) c += sh[qq][4 + 4 * sp + k][lane];
                    b += f.wsp[(size_t)sp * g.n_atm + G.row[k]] * c;
                }
                f.gsun[G.row[k]] = b;
            }
        }
    }
}

// Per-scene tables.  Dependencies: prep -> {segtau -> tinf, tinfg, sunz};
// quadrature tables -> sunz (the direct beam, then the coupling normalisers
// and the source records, in one pass).  st[0] is the scene stream; st[1..3]
// are auxiliary streams forked from it and joined back with events, so the
// independent tables run concurrently.  The quadrature tables (q^sun, the HG
// weights toward the instrument) depend on the view and the asymmetries
// only: `tables` false skips them when the caller knows they are current.
template <typename T>
void launch_sunz(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                 const ViewP &vp) {
    static_assert(kZnBlock == kRayBlock, "the direct beam and the normalisers share the thread layout");
    const dim3 grid((g.nxy + kZnBlock - 1) / kZnBlock, g.nz + 1);
    switch (g.S) {
        case 1: k_sunz<T, 1><<<grid, kZnBlock, 0, st>>>(g, gp, f, vc, vp); break;
        case 2: k_sunz<T, 2><<<grid, kZnBlock, 0, st>>>(g, gp, f, vc, vp); break;
        case 3: k_sunz<T, 3><<<grid, kZnBlock, 0, st>>>(g, gp, f, vc, vp); break;
        default: k_sunz<T, 4><<<grid, kZnBlock, 0, st>>>(g, gp, f, vc, vp); break;
    }
}

template <typename T>
void launch_assemble_pre(cudaStream_t const st[4], cudaEvent_t const ev[5], const GridC &g, const GraphP &gp,
                         const FieldP<T> &f, const ViewC &vc, const ViewP &vp, const SegTab<T> &segtab, bool tables,
                         long long *launches) {
    const int th = 256;
    // ev[0]: start (orders the aux streams after earlier work of the scene stream)
    cudaEventRecord(ev[0], st[0]);
    if (tables) {
        cudaStreamWaitEvent(st[1], ev[0], 0);
        k_tables_cells<T><<<dim3(g.nd, g.S), 128, 0, st[1]>>>(g, f, vc, vp);
        k_tables_norm<T><<<g.S, 128, 0, st[1]>>>(g, f, vc, vp);
        cudaEventRecord(ev[2], st[1]);
    }
    cudaMemsetAsync(f.mus_max_bits, 0, sizeof(unsigned long long), st[0]);
    k_prep<T><<<(g.n_atm + th - 1) / th, th, 0, st[0]>>>(g, f);
    cudaEventRecord(ev[1], st[0]);  // fields ready
    cudaStreamWaitEvent(st[2], ev[1], 0);
    const dim3 sgrid((g.nx + kSegTX - 1) / kSegTX, (g.ny + kSegTY - 1) / kSegTY, g.nz);
    if (segtab.n == 13 && g.R == 1)
        k_segtau_fixed<T, 1, 13><<<sgrid, kSegTX * kSegTY, 0, st[2]>>>(g, f, segtab);
    else if (segtab.n == 49 && g.R == 2)
        k_segtau_fixed<T, 2, 49><<<sgrid, kSegTX * kSegTY, 0, st[2]>>>(g, f, segtab);
    else
        k_segtau<T><<<sgrid, kSegTX * kSegTY, 0, st[2]>>>(g, gp, f);
    k_tinf<T><<<dim3((g.R * g.nxy + th - 1) / th, g.nup), th, 0, st[2]>>>(g, gp, f);
    cudaEventRecord(ev[3], st[2]);
    cudaStreamWaitEvent(st[3], ev[1], 0);
    k_tinfg<T><<<dim3((g.nxy + kRayBlock - 1) / kRayBlock, g.ngd), kRayBlock, 0, st[3]>>>(g, gp, f);
    cudaEventRecord(ev[4], st[3]);
    if (tables) cudaStreamWaitEvent(st[0], ev[2], 0);
    launch_sunz<T>(st[0], g, gp, f, vc, vp);
    cudaStreamWaitEvent(st[0], ev[3], 0);
    cudaStreamWaitEvent(st[0], ev[4], 0);
    if (launches) *launches += tables ? 7 : 5;
}

template <typename T>
void launch_assemble_rows(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                          long long *launches) {
    const int nb = (g.nz + 1) * g.gpl;
    constexpr int W0 = TK_ASM0_W, B0 = TK_ASM0_MINB;
    const size_t sm = asm0_smem<T, W0>(g);
    auto go = [&](auto kern) {
        if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<nb, 32 * W0, sm, st>>>(g, gp, f, vc);
    };
    switch (g.S) {  // the species count as a compile-time constant
        case 1: go(k_asm0<T, 1, W0, B0>); break;
        case 2: go(k_asm0<T, 2, W0, B0>); break;
        case 3: go(k_asm0<T, 3, W0, B0>); break;
        default: go(k_asm0<T, 4, W0, B0>); break;
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
    k_sun<T><<<dim3((g.nxy + kRayBlock - 1) / kRayBlock, g.nz + 1), kRayBlock, 0, st>>>(g, f, vc, vp);
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
                                         const SegTab<T> &, bool, long long *);                                   \
    template void launch_assemble_rows<T>(cudaStream_t, const GridC &, const GraphP &, const FieldP<T> &,         \
                                          const ViewC &, long long *);                                            \
    template void launch_export_csr<T>(cudaStream_t, const GridC &, const GraphP &, const T *, int32_t *,         \
                                       int32_t *, T *, int16_t *, int8_t *);
INST(float)
INST(double)
#undef INST

}  // namespace tk
