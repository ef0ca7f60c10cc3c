// Coupling selection (Sec. 2: the scattering graph keeps the edges with
// C > c_min; Sec. 3: the quadrature cells of Eq. F_term_phase re-drawn among
// the kept directions).  One warp per source node computes the couplings of
// its chains, the kept set, the re-partitioned weights and the routing
// weights, and writes W = q' c for every direction into haloed planes that
// the edge kernel reads at source-relative positions.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "asm_util.cuh"
#include "kern.h"
#include "select.h"

namespace tk {

// max over voxels of the total scattering coefficient, summed over species
// in FP64 (the coupling of a Lambertian node uses A times it)
template <typename T>
__global__ void k_sel_musmax(GridC g, FieldP<T> f, unsigned long long *bits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (i < g.n_atm) {
        for (int sp = 0; sp < g.S; ++sp) m += (double)f.mu_s[(size_t)sp * g.n_atm + i];
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(bits, (unsigned long long)__double_as_longlong(m));
}

// HG of every species toward every lattice point (cell order)
__global__ void k_sel_points(GridC g, ViewC vc, ViewP vp, int M, double *hgpt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const double *s = vp.lattice + 3 * (size_t)p;
    const double mu = vc.s0[0] * s[0] + vc.s0[1] * s[1] + vc.s0[2] * s[2];
    for (int sp = 0; sp < g.S; ++sp) hgpt[(size_t)sp * M + p] = hg<double>(vc.g[sp], mu);
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// total scattering coefficient of voxel i in FP64 (species summed in order)
template <typename T>
__device__ __forceinline__ double mus64(const GridC &g, const FieldP<T> &f, int i) {
    double s = 0.0;
    for (int sp = 0; sp < g.S; ++sp) s += (double)f.mu_s[(size_t)sp * g.n_atm + i];
    return s;
}

constexpr int kSelWarps = 4;

template <typename T>
__global__ void __launch_bounds__(32 * kSelWarps) k_select(GridC g, GraphP gp, FieldP<T> f, ViewC vc, ViewP vp,
                                                          SelP sp, T *w_iso, T *w_sun) {
    __shared__ int s_cnt[kSelWarps][kSelMaxDir];
    __shared__ double s_h[kSelWarps][MAX_SPECIES][kSelMaxDir];
    __shared__ double s_c[kSelWarps][kSelMaxDir];
    __shared__ unsigned char s_kept[kSelWarps][kSelMaxDir];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * kSelWarps + w;
    if (j >= g.n_nodes) return;  // whole warps leave together
    int *cnt = s_cnt[w];
    double *cc = s_c[w];
    unsigned char *kept = s_kept[w];
    const double mus_lamb = vc.albedo * __longlong_as_double((long long)*sp.musmax_bits);
    const bool ground = j >= g.n_atm;
    const int jj = ground ? j - g.n_atm : j;
    const int z = ground ? g.nz : jj / g.nxy, r = jj - (ground ? 0 : z * g.nxy), y = r / g.nx, x = r - y * g.nx;
    const int nd = ground ? g.ngd : g.nd;
    const double mus_src = ground ? mus_lamb : mus64(g, f, j);

    // couplings of the chains and the kept set
    int ndrop = 0;
    for (int u = lane; u < nd; u += 32) {
        double C = -1.0;  // -1: the chain has no receiver
        if (!ground) {
            const int4 d = gp.dirs[u];
            const int rz = z + d.z;
            if (rz < g.nz) {
                double mus_n, dist;
                if (rz >= 0) {
                    const int xn = wrap_small(x + d.x, g.nx), yn = wrap_small(y + d.y, g.ny);
                    mus_n = mus64(g, f, (rz * g.ny + yn) * g.nx + xn);
                    dist = gp.dir_len[u];
                } else {  // the chain hits the ground before its first node
                    mus_n = mus_lamb;
                    dist = ((double)z + 0.5) / (double)(-d.z) * gp.dir_len[u];
                }
                C = sqrt(mus_src * mus_n) / dist;
            }
        } else {
            const int4 m = gp.gmem1[u];
            if ((double)m.z - 0.5 <= (double)g.nz) {
                const int xn = wrap_small(x + m.x, g.nx), yn = wrap_small(y + m.y, g.ny);
                C = sqrt(mus_src * mus64(g, f, ((m.z - 1) * g.ny + yn) * g.nx + xn)) / gp.gdist1[u];
            }
        }
        const bool k = !(sp.c_min > 0.0) || C < 0.0 || C > sp.c_min;
        kept[u] = k;
        cc[u] = C;
        ndrop += !k;
        if (!ground) {
            cnt[u] = k ? vp.cell_start[u + 1] - vp.cell_start[u] : 0;
            for (int s = 0; s < g.S; ++s) s_h[w][s][u] = k ? f.cellsum[s * g.nd + u] : 0.0;
        } else {
            s_h[w][0][u] = k ? sp.gzsum[u] : 0.0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) ndrop += __shfl_xor_sync(0xffffffffu, ndrop, o);
    __syncwarp();

    // the points of every dropped cell join their closest kept direction
    if (ndrop > 0) {
        for (int u = 0; u < nd; ++u) {
            if (kept[u]) continue;
            if (!ground) {
                for (int p = vp.cell_start[u] + lane; p < vp.cell_start[u + 1]; p += 32) {
                    const unsigned char *rk = sp.rank + (size_t)p * nd;
                    int v = -1;
                    for (int q = 1; q < nd; ++q) {
                        const int c = rk[q];
                        if (kept[c]) {
                            v = c;
                            break;
                        }
                    }
                    if (v >= 0) {
                        atomicAdd(&cnt[v], 1);
                        for (int s = 0; s < g.S; ++s) atomicAdd(&s_h[w][s][v], sp.hgpt[(size_t)s * sp.M + p]);
                    }
                }
            } else {
                for (int p = sp.gcell_start[u] + lane; p < sp.gcell_start[u + 1]; p += 32) {
                    const unsigned char *rk = sp.grank + (size_t)p * nd;
                    int v = -1;
                    for (int q = 1; q < nd; ++q) {
                        const int c = rk[q];
                        if (kept[c]) {
                            v = c;
                            break;
                        }
                    }
                    if (v >= 0) atomicAdd(&s_h[w][0][v], sp.gz[p]);
                }
            }
        }
        __syncwarp();
    }

    // weights and routing normalisers over the chains with a receiver
    double wsp[MAX_SPECIES], htot[MAX_SPECIES];
    if (!ground) {
        for (int s = 0; s < g.S; ++s) {
            const double ms = (double)f.mu_s[(size_t)s * g.n_atm + j];
            wsp[s] = mus_src > 0.0 ? ms / mus_src : 1.0 / g.S;
            double t = 0.0;
            for (int u = lane; u < g.nd; u += 32) t += f.cellsum[s * g.nd + u];
            htot[s] = warp_sum_d(t);
        }
    }
    double sq = 0.0, sqc = 0.0, sqs = 0.0, sqcs = 0.0;
    for (int u = lane; u < nd; u += 32) {
        double qi, qs;
        if (!ground) {
            qi = (double)cnt[u] / (double)sp.M;
            qs = 0.0;
            for (int s = 0; s < g.S; ++s) qs += wsp[s] * (s_h[w][s][u] / htot[s]);
        } else {
            qi = s_h[w][0][u] / sp.gztot;
            qs = qi;
        }
        if (cc[u] >= 0.0) {
            sq += qi;
            sqc += qi * cc[u];
            sqs += qs;
            sqcs += qs * cc[u];
        }
    }
    sq = warp_sum_d(sq);
    sqc = warp_sum_d(sqc);
    sqs = warp_sum_d(sqs);
    sqcs = warp_sum_d(sqcs);
    const bool ci_on = vc.coupling && sqc > 0.0, cs_on = vc.coupling && sqcs > 0.0;
    for (int u = lane; u < nd; u += 32) {
        double qi, qs;
        if (!ground) {
            qi = (double)cnt[u] / (double)sp.M;
            qs = 0.0;
            for (int s = 0; s < g.S; ++s) qs += wsp[s] * (s_h[w][s][u] / htot[s]);
        } else {
            qi = s_h[w][0][u] / sp.gztot;
            qs = qi;
        }
        const double C = cc[u];
        const double ci = (ci_on && C >= 0.0) ? C * sq / sqc : 1.0;
        const double cs = (cs_on && C >= 0.0) ? C * sqs / sqcs : 1.0;
        store_halo(w_iso + (size_t)u * g.npad, g, x, y, z, (T)(qi * ci));
        store_halo(w_sun + (size_t)u * g.npad, g, x, y, z, (T)(qs * cs));
    }
}

template <typename T>
void launch_select(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                   const ViewP &vp, const SelP &sp, T *w_iso, T *w_sun, long long *launches) {
    cudaMemsetAsync(sp.musmax_bits, 0, sizeof(unsigned long long), st);
    k_sel_musmax<T><<<(g.n_atm + 255) / 256, 256, 0, st>>>(g, f, sp.musmax_bits);
    k_sel_points<<<(sp.M + 127) / 128, 128, 0, st>>>(g, vc, vp, sp.M, sp.hgpt);
    k_select<T><<<(g.n_nodes + kSelWarps - 1) / kSelWarps, 32 * kSelWarps, 0, st>>>(g, gp, f, vc, vp, sp, w_iso,
                                                                                     w_sun);
    if (launches) *launches += 3;
}

template void launch_select<float>(cudaStream_t, const GridC &, const GraphP &, const FieldP<float> &, const ViewC &,
                                   const ViewP &, const SelP &, float *, float *, long long *);
template void launch_select<double>(cudaStream_t, const GridC &, const GraphP &, const FieldP<double> &,
                                    const ViewC &, const ViewP &, const SelP &, double *, double *, long long *);

}  // namespace tk
