// Coupling selection (Sec. 2: the scattering graph keeps the edges with
// C > c_min; Sec. 3: the quadrature cells of Eq. F_term_phase re-drawn among
// the kept directions).  One warp per source node computes the couplings of
// its chains, the kept set, the re-partitioned weights and the routing
// weights, and writes W = q' c for every direction into haloed planes that
// the edge kernel reads at source-relative positions.
#include <cuda_runtime.h>

#include <algorithm>
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

// HG of every species toward every lattice point (in the order of the rankings)
__global__ void k_sel_points(GridC g, ViewC vc, const double *lat, int M, double *hgpt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const double *s = lat + 3 * (size_t)p;
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

constexpr int kSelWarps = 8;
// kept directions up to which a point's target comes from cosines over the
// kept list rather than from its ranking
constexpr int kSelDots = 12;

// Per-scene constants of the re-partition in the compute type: the HG
// weight of every lattice point, the HG sum of every cell and each species'
// total (the denominator of q^sun).
template <typename T>
__global__ void k_sel_consts(GridC g, SelP sp, const double *cellsum, T *hgpt_t, T *cellsum_t, T *htot_t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.S * sp.M) hgpt_t[i] = (T)sp.hgpt[i];
    if (i < g.S * g.nd) cellsum_t[i] = (T)cellsum[i];
    if (i < g.S) {
        double t = 0.0;
        for (int u = 0; u < g.nd; ++u) t += cellsum[i * g.nd + u];
        htot_t[i] = (T)t;
    }
}

// The source of a selection warp and its total scattering coefficient: FP64
// on FP64 scenes; FP32 scenes take the FP32 sum and the FP64 one only near
// the threshold.
template <typename T>
struct SelSrc {
    bool ground;
    int j, x, y, z, nd;
    double mus_lamb, mus_src64;
    T mus_src;
};
template <typename T>
__device__ __forceinline__ SelSrc<T> sel_src(const GridC &g, const FieldP<T> &f, const ViewC &vc, const SelP &sp,
                                             int j) {
    SelSrc<T> o;
    o.j = j;
    o.mus_lamb = vc.albedo * __longlong_as_double((long long)*sp.musmax_bits);
    o.ground = j >= g.n_atm;
    const int jj = o.ground ? j - g.n_atm : j;
    o.z = o.ground ? g.nz : jj / g.nxy;
    const int r = jj - (o.ground ? 0 : o.z * g.nxy);
    o.y = r / g.nx;
    o.x = r - o.y * g.nx;
    o.nd = o.ground ? g.ngd : g.nd;
    o.mus_src64 = (sizeof(T) == 8) ? (o.ground ? o.mus_lamb : mus64(g, f, j)) : 0.0;
    o.mus_src = (sizeof(T) == 8) ? (T)o.mus_src64 : (o.ground ? (T)o.mus_lamb : f.mu_st[j]);
    return o;
}

// The coupling C of chain u of the source (-1: the chain has no receiver) and
// whether the chain is kept (always, without a receiver).
template <typename T>
__device__ __forceinline__ void sel_chain(const GridC &g, const GraphP &gp, const FieldP<T> &f, const SelP &sp,
                                          const SelSrc<T> &src, int u, T &C, bool &keep) {
    C = T(-1);
    keep = true;
    int nidx = -1;  // receiver voxel (-1: the ground)
    bool recv = false;
    T dist = T(1);
    const int x = src.x, y = src.y, z = src.z;
    if (!src.ground) {
        const int4 d = gp.dirs[u];
        const int rz = z + d.z;
        if (rz < g.nz) {
            recv = true;
            if (rz >= 0) {
                const int xn = wrap_small(x + d.x, g.nx), yn = wrap_small(y + d.y, g.ny);
                nidx = (rz * g.ny + yn) * g.nx + xn;
                dist = Cst<T>::dir_len(gp, u);
            } else {  // the chain hits the ground before its first node
                dist = ((T)z + T(0.5)) / (T)(-d.z) * Cst<T>::dir_len(gp, u);
            }
        }
    } else {
        const int4 m = gp.gmem1[u];
        if ((double)m.z - 0.5 <= (double)g.nz) {
            recv = true;
            const int xn = wrap_small(x + m.x, g.nx), yn = wrap_small(y + m.y, g.ny);
            nidx = ((m.z - 1) * g.ny + yn) * g.nx + xn;
            dist = Cst<T>::gdist1(gp, u);
        }
    }
    // the FP64 distance to the first receiver (the oracle's arithmetic)
    auto dist64 = [&]() -> double {
        if (src.ground) return gp.gdist1[u];
        const int dz = gp.dirs[u].z;
        return z + dz >= 0 ? gp.dir_len[u] : ((double)z + 0.5) / (double)(-dz) * gp.dir_len[u];
    };
    if (recv) {
        if constexpr (sizeof(T) == 4) {
            // FP32 value (relative error below 1e-6); the FP64 coupling
            // decides only where the FP32 one is that close to c_min
            const float mus_n = nidx >= 0 ? f.mu_st[nidx] : (float)src.mus_lamb;
            const float c32 = sqrtf(src.mus_src * mus_n) / dist;
            C = c32;
            if (sp.c_min > 0.0) {
                if (fabs((double)c32 - sp.c_min) > 1e-5 * sp.c_min) {
                    keep = (double)c32 > sp.c_min;
                } else {
                    const double ms = src.ground ? src.mus_lamb : mus64(g, f, src.j);
                    const double mn = nidx >= 0 ? mus64(g, f, nidx) : src.mus_lamb;
                    keep = sqrt(ms * mn) / dist64() > sp.c_min;
                }
            }
        } else {
            const double mn = nidx >= 0 ? mus64(g, f, nidx) : src.mus_lamb;
            C = sqrt(src.mus_src64 * mn) / dist64();
            keep = !(sp.c_min > 0.0) || C > sp.c_min;
        }
    }
}

// Which directions a source keeps (bit u of its mask) fixes how its lattice
// points are re-drawn: the re-partition is a function of the kept set (and of
// whether the source is a ground node) alone, so it is computed once per
// distinct kept set.  Pass 1 (one thread per source, so that the threads of
// a warp gather the first receivers of one direction from consecutive
// voxels): the mask, and whether the source has anything to re-draw (some
// direction dropped and some kept): rep = -2 if so, else -1.
template <typename T>
__global__ void k_sel_mask(GridC g, GraphP gp, FieldP<T> f, ViewC vc, SelP sp) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_nodes) return;
    const SelSrc<T> src = sel_src(g, f, vc, sp, j);
    unsigned long long m0 = 0ull, m1 = 0ull;
    int nl = 0, nk = 0;
    for (int u = 0; u < src.nd; ++u) {
        T C;
        bool keep;
        sel_chain(g, gp, f, sp, src, u, C, keep);
        if (keep) {
            if (u < 64) m0 |= 1ull << u;
            else m1 |= 1ull << (u - 64);
            ++nk;
        } else {
            ++nl;
        }
    }
    sp.mask[j] = make_ulonglong2(m0, m1);
    sp.rep[j] = (nl > 0 && nk > 0) ? -2 : -1;
}

__device__ __forceinline__ unsigned sel_hash(unsigned long long a, unsigned long long b, bool ground) {
    unsigned long long h = a * 0x9E3779B97F4A7C15ull;
    h ^= (b + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full;
    h ^= ground ? 0xD6E8FEB86659FD93ull : 0ull;
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 32;
    return (unsigned)h;
}

// Pass 2 (one thread per source with something to re-draw): the first source
// of each distinct (kept set, ground) to claim a slot of the open-addressing
// table becomes its representative; every other source finds it by linear
// probing.  Which source wins depends on timing, but the re-partition it
// computes is the same function of the kept set, so the weights are too.
// The table has at least twice as many slots as sources and is cleared
// before the pass, so a free slot is always found.
__global__ void k_sel_dedupe(int n, int n_atm, SelP sp) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || sp.rep[j] != -2) return;
    const ulonglong2 m = sp.mask[j];
    const bool ground = j >= n_atm;
    unsigned h = sel_hash(m.x, m.y, ground) & (unsigned)(sp.ht - 1);
    for (int probe = 0; probe < sp.ht; ++probe) {
        const int old = atomicCAS(sp.table + h, -1, j);
        if (old == -1) {
            sp.rep[j] = j;
            sp.rlist[atomicAdd(sp.rcount, 1)] = j;
            return;
        }
        const ulonglong2 mo = sp.mask[old];
        if (mo.x == m.x && mo.y == m.y && (old >= n_atm) == ground) {
            sp.rep[j] = old;
            return;
        }
        h = (h + 1) & (unsigned)(sp.ht - 1);
    }
}

// Pass 3 (a block of kSelWarps warps per representative source; persistent
// blocks take the representatives from the list one after another): the
// points of every dropped cell join their closest kept direction; the point
// counts and the HG sums of every direction after the re-draw go to pcnt /
// ph of the representative.  The values (sums) are in the compute type T;
// the decisions (which kept direction a point joins) are exact.
template <typename T>
__global__ void __launch_bounds__(32 * kSelWarps) k_sel_part(GridC g, ViewP vp, SelP sp, const T *hgpt,
                                                            const T *cellsum) {
    __shared__ int s_cnt[kSelWarps][kSelMaxDir];
    __shared__ T s_h[kSelWarps][MAX_SPECIES][kSelMaxDir];
    __shared__ unsigned char s_kept[kSelMaxDir];
    __shared__ unsigned char s_list[kSelMaxDir];
    __shared__ unsigned char s_klist[kSelMaxDir];
    __shared__ int s_r, s_nl, s_nk;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    constexpr int NT = 32 * kSelWarps;
    const int nrep = sp.rcount[0];
    for (;;) {
        if (tid == 0) s_r = atomicAdd(sp.rcount + 1, 1);
        __syncthreads();
        const int ri = s_r;
        if (ri >= nrep) break;
        const int j = sp.rlist[ri];
        const bool ground = j >= g.n_atm;
        const int nd = ground ? g.ngd : g.nd;
        const ulonglong2 mk = sp.mask[j];
        // every warp's accumulators: the kept cells' own points in warp 0's
        for (int u = tid; u < nd; u += NT) {
            const bool keep = ((u < 64 ? mk.x >> u : mk.y >> (u - 64)) & 1ull) != 0ull;
            s_kept[u] = keep;
            for (int q = 0; q < kSelWarps; ++q) {
                const bool own = q == 0 && keep;
                s_cnt[q][u] = (!ground && own) ? vp.cell_start[u + 1] - vp.cell_start[u] : 0;
                if (!ground) {
                    for (int s = 0; s < g.S; ++s) s_h[q][s][u] = own ? cellsum[s * g.nd + u] : T(0);
                } else {
                    s_h[q][0][u] = own ? (T)sp.gzsum[u] : T(0);
                }
            }
        }
        __syncthreads();
        if (w == 0) {  // the dropped and the kept directions, in order
            int nl = 0, nk = 0;
            for (int b = 0; b < nd; b += 32) {
                const int u = b + lane;
                const bool dr = u < nd && !s_kept[u], kp = u < nd && s_kept[u];
                const unsigned m = __ballot_sync(0xffffffffu, dr), mkb = __ballot_sync(0xffffffffu, kp);
                const unsigned below = (1u << lane) - 1u;
                if (dr) s_list[nl + __popc(m & below)] = (unsigned char)u;
                if (kp) s_klist[nk + __popc(mkb & below)] = (unsigned char)u;
                nl += __popc(m);
                nk += __popc(mkb);
            }
            if (lane == 0) {
                s_nl = nl;
                s_nk = nk;
            }
        }
        __syncthreads();
        const int nl = s_nl, nk = s_nk;
        int *cnt = s_cnt[w];
        // The points of the dropped cells, cell after cell, are dealt to the
        // block's threads round robin (thread t takes points t, t + NT, ...
        // of that sequence), so every thread has work whatever the number of
        // dropped cells.  Inside a cell the points are ordered by their
        // rankings, so a thread's target changes rarely and it adds a run at
        // a time into its warp's accumulators.  With many kept directions a
        // point's target is the first kept one in its ranking; with few, the
        // largest FP32 cosine over the kept list picks it, and exact FP64
        // cosines (the ranking's arithmetic) decide near-ties.
        {
            const unsigned char *rk = ground ? sp.grank : sp.rank;
            const int *cs = ground ? sp.gcell_start : vp.cell_start;
            const float4 *pf = ground ? sp.glatf : sp.latf;
            const double *pd = ground ? sp.glat : sp.lat;
            const float4 *df = sp.dirf + (ground ? g.nd : 0);
            const double *dd = vp.dirhat + 3 * (ground ? g.nd : 0);
            const bool dots = nk <= kSelDots;
            int tot = 0;  // points of the dropped cells
            for (int i = 0; i < nl; ++i) tot += cs[s_list[i] + 1] - cs[s_list[i]];
            int ci = 0, off = tid;  // the thread's cell (index into the list) and point offset inside it
            int cur = -1, n = 0;
            T a[MAX_SPECIES] = {T(0), T(0), T(0), T(0)};
            for (int f0 = tid; f0 < tot; f0 += NT) {
                int csz = cs[s_list[ci] + 1] - cs[s_list[ci]];
                while (off >= csz) {
                    off -= csz;
                    ++ci;
                    csz = cs[s_list[ci] + 1] - cs[s_list[ci]];
                }
                const int p = cs[s_list[ci]] + off;
                off += NT;
                int v = -1;
                if (dots) {
                    const float4 pt = pf[p];
                    float b1 = -3.f, b2 = -3.f;
                    for (int t = 0; t < nk; ++t) {
                        const int c = s_klist[t];
                        const float4 d = df[c];
                        const float co = d.x * pt.x + d.y * pt.y + d.z * pt.z;
                        if (co > b1) {
                            b2 = b1;
                            b1 = co;
                            v = c;
                        } else if (co > b2) {
                            b2 = co;
                        }
                    }
                    if (b1 - b2 <= 4e-6f) {
                        const double *q3 = pd + 3 * (size_t)p;
                        double best = -3.0;
                        for (int t = 0; t < nk; ++t) {
                            const int c = s_klist[t];
                            const double *h3 = dd + 3 * c;
                            const double co = __dadd_rn(__dadd_rn(__dmul_rn(h3[0], q3[0]), __dmul_rn(h3[1], q3[1])),
                                                        __dmul_rn(h3[2], q3[2]));
                            if (co > best) {
                                best = co;
                                v = c;
                            }
                        }
                    }
                } else {
                    const unsigned char *row = rk + (size_t)p * nd;
                    for (int q = 1; q < nd; ++q) {
                        const int c = row[q];
                        if (s_kept[c]) {
                            v = c;
                            break;
                        }
                    }
                }
                if (v != cur) {
                    if (cur >= 0) {
                        if (!ground) atomicAdd(&cnt[cur], n);
                        for (int s = 0; s < (ground ? 1 : g.S); ++s) atomicAdd(&s_h[w][s][cur], a[s]);
                    }
                    cur = v;
                    n = 0;
                    for (int s = 0; s < MAX_SPECIES; ++s) a[s] = T(0);
                }
                ++n;
                if (ground) {
                    a[0] += (T)sp.gz[p];
                } else {
                    for (int s = 0; s < g.S; ++s) a[s] += hgpt[(size_t)s * sp.M + p];
                }
            }
            if (cur >= 0) {
                if (!ground) atomicAdd(&cnt[cur], n);
                for (int s = 0; s < (ground ? 1 : g.S); ++s) atomicAdd(&s_h[w][s][cur], a[s]);
            }
        }
        __syncthreads();
        // the warps' accumulators summed in a fixed order
        T *ph = reinterpret_cast<T *>(sp.ph) + (size_t)j * g.S * sp.dmax;
        for (int u = tid; u < nd; u += NT) {
            int c = 0;
            for (int q = 0; q < kSelWarps; ++q) c += s_cnt[q][u];
            sp.pcnt[(size_t)j * sp.dmax + u] = c;
            for (int s = 0; s < (ground ? 1 : g.S); ++s) {
                T hsum = T(0);
                for (int q = 0; q < kSelWarps; ++q) hsum += s_h[q][s][u];
                ph[(size_t)s * sp.dmax + u] = hsum;
            }
        }
        __syncthreads();  // the shared arrays are reused for the next representative
    }
}

// Pass 4 (one thread per source): the weights and routing normalisers over
// the chains with a receiver, from the source's couplings and its kept set's
// re-partition (the representative's, or the cells themselves when nothing
// was re-drawn), into the haloed planes W = q' c.  The first sweep over the
// directions sums the normalisers, the second forms the weights again and
// stores them (the threads of a warp store one direction's plane at
// consecutive voxels).
template <typename T>
struct SelQ {
    T qi, qs, C;
};
template <typename T>
__device__ __forceinline__ SelQ<T> sel_q(const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewP &vp,
                                         const SelP &sp, const SelSrc<T> &src, int rep, const T *ph, const T *cellsum,
                                         const T (&wsp)[MAX_SPECIES], const T (&rht)[MAX_SPECIES], T rM, T rz, int u) {
    SelQ<T> o;
    bool keep;
    sel_chain(g, gp, f, sp, src, u, o.C, keep);
    o.qi = T(0);
    o.qs = T(0);
    if (!src.ground) {
        int cnt;
        T h[MAX_SPECIES];
        if (ph) {
            cnt = sp.pcnt[(size_t)rep * sp.dmax + u];
            for (int s = 0; s < g.S; ++s) h[s] = ph[(size_t)s * sp.dmax + u];
        } else {
            cnt = keep ? vp.cell_start[u + 1] - vp.cell_start[u] : 0;
            for (int s = 0; s < g.S; ++s) h[s] = keep ? cellsum[s * g.nd + u] : T(0);
        }
        o.qi = (T)cnt * rM;
        for (int s = 0; s < g.S; ++s) o.qs += wsp[s] * (h[s] * rht[s]);
    } else {
        const T h0 = ph ? ph[u] : (keep ? (T)sp.gzsum[u] : T(0));
        o.qi = h0 * rz;
        o.qs = o.qi;
    }
    return o;
}

template <typename T>
__global__ void k_select(GridC g, GraphP gp, FieldP<T> f, ViewC vc, ViewP vp, SelP sp, const T *cellsum,
                         const T *htot_g, T *w_iso, T *w_sun) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n_nodes) return;
    const SelSrc<T> src = sel_src(g, f, vc, sp, j);
    const int nd = src.nd;
    const int rep = sp.rep[j];
    const T *ph = rep >= 0 ? reinterpret_cast<const T *>(sp.ph) + (size_t)rep * g.S * sp.dmax : nullptr;
    T wsp[MAX_SPECIES] = {T(0), T(0), T(0), T(0)}, rht[MAX_SPECIES] = {T(0), T(0), T(0), T(0)};
    if (!src.ground) {
        for (int s = 0; s < g.S; ++s) {
            if constexpr (sizeof(T) == 8) {
                const double ms = (double)f.mu_s[(size_t)s * g.n_atm + j];
                wsp[s] = src.mus_src64 > 0.0 ? ms / src.mus_src64 : 1.0 / g.S;
            } else {
                wsp[s] = f.wsp[(size_t)s * g.n_atm + j];
            }
            rht[s] = T(1) / htot_g[s];
        }
    }
    const T rM = T(1) / (T)sp.M, rz = T(1) / (T)sp.gztot;
    T sq = 0, sqc = 0, sqs = 0, sqcs = 0;
    for (int u = 0; u < nd; ++u) {
        const SelQ<T> o = sel_q(g, gp, f, vp, sp, src, rep, ph, cellsum, wsp, rht, rM, rz, u);
        if (o.C >= T(0)) {
            sq += o.qi;
            sqc += o.qi * o.C;
            sqs += o.qs;
            sqcs += o.qs * o.C;
        }
    }
    const bool ci_on = vc.coupling && sqc > T(0), cs_on = vc.coupling && sqcs > T(0);
    const T fi = ci_on ? sq / sqc : T(0), fs = cs_on ? sqs / sqcs : T(0);
    for (int u = 0; u < nd; ++u) {
        const SelQ<T> o = sel_q(g, gp, f, vp, sp, src, rep, ph, cellsum, wsp, rht, rM, rz, u);
        const T ci = (ci_on && o.C >= T(0)) ? o.C * fi : T(1);
        const T cs = (cs_on && o.C >= T(0)) ? o.C * fs : T(1);
        store_halo(w_iso + (size_t)u * g.npad, g, src.x, src.y, src.z, o.qi * ci);
        store_halo(w_sun + (size_t)u * g.npad, g, src.x, src.y, src.z, o.qs * cs);
    }
}

template <typename T>
void launch_select(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                   const ViewP &vp, const SelP &sp, T *w_iso, T *w_sun, long long *launches) {
    // per-scene constants in the compute type live at the end of hgpt
    T *hgpt_t = reinterpret_cast<T *>(sp.hgpt + (size_t)g.S * sp.M);
    T *cellsum_t = hgpt_t + (size_t)g.S * sp.M;
    T *htot_t = cellsum_t + (size_t)g.S * g.nd;
    cudaMemsetAsync(sp.musmax_bits, 0, sizeof(unsigned long long), st);
    k_sel_musmax<T><<<(g.n_atm + 255) / 256, 256, 0, st>>>(g, f, sp.musmax_bits);
    k_sel_points<<<(sp.M + 127) / 128, 128, 0, st>>>(g, vc, sp.lat, sp.M, sp.hgpt);
    const int nc = std::max(g.S * sp.M, g.S * g.nd);
    k_sel_consts<T><<<(nc + 255) / 256, 256, 0, st>>>(g, sp, f.cellsum, hgpt_t, cellsum_t, htot_t);
    const int nbw = (g.n_nodes + kSelWarps - 1) / kSelWarps, nbt = (g.n_nodes + 127) / 128;
    k_sel_mask<T><<<nbt, 128, 0, st>>>(g, gp, f, vc, sp);
    cudaMemsetAsync(sp.table, 0xff, (size_t)sp.ht * sizeof(int), st);
    cudaMemsetAsync(sp.rcount, 0, 2 * sizeof(int), st);
    k_sel_dedupe<<<(g.n_nodes + 255) / 256, 256, 0, st>>>(g.n_nodes, g.n_atm, sp);
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int nbp = std::max(1, std::min(nbw, 8 * std::max(1, sms)));
        k_sel_part<T><<<nbp, 32 * kSelWarps, 0, st>>>(g, vp, sp, hgpt_t, cellsum_t);
    }
    k_select<T><<<nbt, 128, 0, st>>>(g, gp, f, vc, vp, sp, cellsum_t, htot_t, w_iso, w_sun);
    if (launches) *launches += 7;
}

// ---------------------------------------------------------------------------
// The preselected maximum number of couplings (Sec. 3): the threshold that
// keeps the K largest couplings is the (K + 1)-th largest coupling over every
// chain that has a receiver.  Each chain's coupling is formed once in FP64
// with the arithmetic of the selection's FP64 decision above (FP64 species
// sums, sqrt(mu_s(src) mu_s(n1)) / d), and its bit pattern (a non-negative
// double orders like its bits) plus one is the chain's key (0: no
// receiver).  A radix select finds the key of rank K + 1 from the top in
// passes of kTopkBits bits: every pass histograms, over the keys that share
// the prefix found so far, the next digit; the host picks the digit that
// holds the wanted rank.  Keys are [n_atm][nd] then [n_ground][ngd].
// The receiver of chain e ([n_atm][nd], then [n_ground][ngd]) and its
// source: whether it has one, the receiver voxel (-1: the ground) and the
// FP64 distance to it.
struct TopkChain {
    int j, nidx;
    bool ground, recv;
    double dist;
};
__device__ __forceinline__ TopkChain topk_chain(const GridC &g, const GraphP &gp, long long e) {
    TopkChain c;
    const long long na_ch = (long long)g.n_atm * g.nd;
    c.ground = e >= na_ch;
    int u;
    if (!c.ground) {
        c.j = (int)(e / g.nd);
        u = (int)(e - (long long)c.j * g.nd);
    } else {
        const long long q = e - na_ch;
        c.j = (int)(q / g.ngd);
        u = (int)(q - (long long)c.j * g.ngd);
    }
    const int z = c.ground ? g.nz : c.j / g.nxy, r = c.ground ? c.j : c.j - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    c.recv = false;
    c.nidx = -1;
    c.dist = 1.0;
    if (!c.ground) {
        const int4 d = gp.dirs[u];
        const int rz = z + d.z;
        if (rz < g.nz) {
            c.recv = true;
            if (rz >= 0) {
                c.nidx = (rz * g.ny + wrap_small(y + d.y, g.ny)) * g.nx + wrap_small(x + d.x, g.nx);
                c.dist = gp.dir_len[u];
            } else {
                c.dist = ((double)z + 0.5) / (double)(-d.z) * gp.dir_len[u];
            }
        }
    } else {
        const int4 m = gp.gmem1[u];
        if ((double)m.z - 0.5 <= (double)g.nz) {
            c.recv = true;
            c.nidx = ((m.z - 1) * g.ny + wrap_small(y + m.y, g.ny)) * g.nx + wrap_small(x + m.x, g.nx);
            c.dist = gp.gdist1[u];
        }
    }
    return c;
}

// the exact key of chain e: 1 + the bits of its FP64 coupling (0: no receiver)
template <typename T>
__device__ __forceinline__ unsigned long long topk_key64(const GridC &g, const GraphP &gp, const FieldP<T> &f,
                                                         double mus_lamb, long long e) {
    const TopkChain c = topk_chain(g, gp, e);
    if (!c.recv) return 0ull;
    const double ms = c.ground ? mus_lamb : mus64(g, f, c.j);
    const double mn = c.nidx >= 0 ? mus64(g, f, c.nidx) : mus_lamb;
    return (unsigned long long)__double_as_longlong(sqrt(ms * mn) / c.dist) + 1ull;
}

template <typename T>
__global__ void k_topk_keys(GridC g, GraphP gp, FieldP<T> f, ViewC vc, const unsigned long long *musmax_bits,
                            unsigned long long *keys) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)g.n_atm * g.nd + (long long)g.n_ground * g.ngd;
    if (e >= tot) return;
    const double mus_lamb = vc.albedo * __longlong_as_double((long long)*musmax_bits);
    keys[e] = topk_key64(g, gp, f, mus_lamb, e);
}

// The same couplings in FP32 (relative error of a few 1e-7 against the FP64
// ones): 1 + the bits of the FP32 value (0: no receiver).
template <typename T>
__global__ void k_topk_keys32(GridC g, GraphP gp, FieldP<T> f, ViewC vc, const unsigned long long *musmax_bits,
                              unsigned int *keys) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)g.n_atm * g.nd + (long long)g.n_ground * g.ngd;
    if (e >= tot) return;
    const float mus_lamb = (float)(vc.albedo * __longlong_as_double((long long)*musmax_bits));
    const TopkChain c = topk_chain(g, gp, e);
    unsigned int key = 0u;
    if (c.recv) {
        const float ms = c.ground ? mus_lamb : (float)f.mu_st[c.j];
        const float mn = c.nidx >= 0 ? (float)f.mu_st[c.nidx] : mus_lamb;
        key = (unsigned int)__float_as_int(sqrtf(ms * mn) / (float)c.dist) + 1u;
    }
    keys[e] = key;
}

// The chains whose FP32 coupling lies in [lo, hi] (their indices appended to
// band in any order) and the number of chains above hi.
__global__ void k_topk_band(const unsigned int *__restrict__ keys, long long n, double lo, double hi, int *band,
                            int *counts) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned int k = keys[i];
        if (k == 0u) continue;
        const double c = (double)__int_as_float((int)(k - 1u));
        if (c > hi)
            atomicAdd(counts + 1, 1);
        else if (c >= lo)
            band[atomicAdd(counts, 1)] = (int)i;
    }
}

// exact keys of the band's chains
template <typename T>
__global__ void k_topk_band_keys(GridC g, GraphP gp, FieldP<T> f, ViewC vc, const unsigned long long *musmax_bits,
                                 const int *band, int nb, unsigned long long *keys) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const double mus_lamb = vc.albedo * __longlong_as_double((long long)*musmax_bits);
    keys[i] = topk_key64(g, gp, f, mus_lamb, band[i]);
}

constexpr int kTopkBits = 11;

// histogram of digit (key >> shift) & mask over the keys whose bits above
// shift + kTopkBits equal prefix (pass 0: every key that has a receiver)
__global__ void k_topk_hist(const unsigned long long *__restrict__ keys, long long n, int shift, int width,
                            int hi_shift, unsigned long long prefix, unsigned int *hist) {
    __shared__ unsigned int h[1 << kTopkBits];
    for (int b = threadIdx.x; b < (1 << kTopkBits); b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const unsigned long long mask = (1ull << width) - 1ull;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        if (k == 0ull) continue;
        if (hi_shift < 64 && (k >> hi_shift) != prefix) continue;
        atomicAdd(&h[(k >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < (1 << kTopkBits); b += blockDim.x)
        if (h[b]) atomicAdd(hist + b, h[b]);
}

// the same histogram over 32-bit keys (the FP32 couplings)
__global__ void k_topk_hist32(const unsigned int *__restrict__ keys, long long n, int shift, int width, int hi_shift,
                              unsigned int prefix, unsigned int *hist) {
    __shared__ unsigned int h[1 << kTopkBits];
    for (int b = threadIdx.x; b < (1 << kTopkBits); b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const unsigned int mask = (1u << width) - 1u;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned int k = keys[i];
        if (k == 0u) continue;
        if (hi_shift < 32 && (k >> hi_shift) != prefix) continue;
        atomicAdd(&h[(k >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < (1 << kTopkBits); b += blockDim.x)
        if (h[b]) atomicAdd(hist + b, h[b]);
}

template <typename T>
void launch_topk_keys32(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                        unsigned long long *musmax_bits, unsigned int *keys, long long *launches) {
    const long long tot = (long long)g.n_atm * g.nd + (long long)g.n_ground * g.ngd;
    cudaMemsetAsync(musmax_bits, 0, sizeof(unsigned long long), st);
    k_sel_musmax<T><<<(g.n_atm + 255) / 256, 256, 0, st>>>(g, f, musmax_bits);
    k_topk_keys32<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(g, gp, f, vc, musmax_bits, keys);
    if (launches) *launches += 2;
}

void launch_topk_hist32(cudaStream_t st, const unsigned int *keys, long long n, int shift, int width, int hi_shift,
                        unsigned int prefix, unsigned int *hist, int nblocks) {
    cudaMemsetAsync(hist, 0, sizeof(unsigned int) << kTopkBits, st);
    k_topk_hist32<<<nblocks, 256, 0, st>>>(keys, n, shift, width < kTopkBits ? width : kTopkBits, hi_shift, prefix,
                                           hist);
}

void launch_topk_band(cudaStream_t st, const unsigned int *keys, long long n, double lo, double hi, int *band,
                      int *counts, int nblocks) {
    cudaMemsetAsync(counts, 0, 2 * sizeof(int), st);
    k_topk_band<<<nblocks, 256, 0, st>>>(keys, n, lo, hi, band, counts);
}

template <typename T>
void launch_topk_band_keys(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                           const unsigned long long *musmax_bits, const int *band, int nb, unsigned long long *keys) {
    if (nb > 0) k_topk_band_keys<T><<<(nb + 255) / 256, 256, 0, st>>>(g, gp, f, vc, musmax_bits, band, nb, keys);
}

template <typename T>
void launch_topk_keys(cudaStream_t st, const GridC &g, const GraphP &gp, const FieldP<T> &f, const ViewC &vc,
                      unsigned long long *musmax_bits, unsigned long long *keys, long long *launches) {
    const long long tot = (long long)g.n_atm * g.nd + (long long)g.n_ground * g.ngd;
    cudaMemsetAsync(musmax_bits, 0, sizeof(unsigned long long), st);
    k_sel_musmax<T><<<(g.n_atm + 255) / 256, 256, 0, st>>>(g, f, musmax_bits);
    k_topk_keys<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(g, gp, f, vc, musmax_bits, keys);
    if (launches) *launches += 2;
}

void launch_topk_hist(cudaStream_t st, const unsigned long long *keys, long long n, int shift, int width,
                      int hi_shift, unsigned long long prefix, unsigned int *hist, int nblocks) {
    cudaMemsetAsync(hist, 0, sizeof(unsigned int) << kTopkBits, st);
    k_topk_hist<<<nblocks, 256, 0, st>>>(keys, n, shift, width < kTopkBits ? width : kTopkBits, hi_shift, prefix,
                                         hist);
}

template void launch_topk_keys<float>(cudaStream_t, const GridC &, const GraphP &, const FieldP<float> &,
                                      const ViewC &, unsigned long long *, unsigned long long *, long long *);
template void launch_topk_keys32<float>(cudaStream_t, const GridC &, const GraphP &, const FieldP<float> &,
                                        const ViewC &, unsigned long long *, unsigned int *, long long *);
template void launch_topk_keys32<double>(cudaStream_t, const GridC &, const GraphP &, const FieldP<double> &,
                                         const ViewC &, unsigned long long *, unsigned int *, long long *);
template void launch_topk_band_keys<float>(cudaStream_t, const GridC &, const GraphP &, const FieldP<float> &,
                                           const ViewC &, const unsigned long long *, const int *, int,
                                           unsigned long long *);
template void launch_topk_band_keys<double>(cudaStream_t, const GridC &, const GraphP &, const FieldP<double> &,
                                            const ViewC &, const unsigned long long *, const int *, int,
                                            unsigned long long *);
template void launch_topk_keys<double>(cudaStream_t, const GridC &, const GraphP &, const FieldP<double> &,
                                       const ViewC &, unsigned long long *, unsigned long long *, long long *);

template void launch_select<float>(cudaStream_t, const GridC &, const GraphP &, const FieldP<float> &, const ViewC &,
                                   const ViewP &, const SelP &, float *, float *, long long *);
template void launch_select<double>(cudaStream_t, const GridC &, const GraphP &, const FieldP<double> &,
                                    const ViewC &, const ViewP &, const SelP &, double *, double *, long long *);

}  // namespace tk
