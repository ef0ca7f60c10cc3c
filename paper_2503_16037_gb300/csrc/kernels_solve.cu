// Solver kernels for (I - K) x = s (Eq. flux_system of Mikkonen et al.;
// the Neumann / source iteration is the series of Eq. fs_sum).
//
// The sweeps walk rows of receivers (K in CSR order by row) in groups of 128
// rows; the column of each slot comes from the row template of the row's
// layer instead of a stored index, so only the 4-byte values stream.
// Reductions are deterministic: fixed grids, fixed per-block order,
// fixed-order trees.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "kern.h"
#include "batch.h"
#include "stage.cuh"

namespace tk {

// ---- Row-group kernels.  One pass over K does one of the operations below
// (an "Op"): it accumulates, for each row of a group, the products of the
// row's values with the source values it gathers, and finishes the row
// (combination of the warps' partial sums in a fixed order, the row update,
// per-group partial sums of squares).  The plain driver runs one block of W
// warps per group and reads the values directly; for FP32 ops that gather
// from FP32 vectors it first copies the group's source rows into a
// shared-memory tile (k_tile); the pipelined driver (k_pipe) streams the
// values through shared memory.  Source values are gathered from haloed
// vectors (the template offset is the only index arithmetic), and every row
// result is stored with its halo copies.

// Op interface (both drivers): A / NA: accumulator type and words per lane;
// kPart: the op writes per-row-block partial sums part[4 gi + k]; Pre: the
// epilogue inputs of one row, loaded when a group starts (pre) so that their
// latency hides behind the group's slots; slot / add: per-slot constants and
// the accumulation of one value times one gathered source value;
// combine_row: the words of row k summed over the W warps in a fixed order;
// finish_row: the row update, returning the row's share of the partial sum.

// The refinement update x += d (with the FP32-pair split of x when xh is
// set), done row by row in the epilogue of the pass that produces d
// (x == nullptr: none); the same arithmetic as k_update_x.
struct XUpd {
    double *x = nullptr;
    float *xh = nullptr, *xl = nullptr;
    template <typename T>
    __device__ __forceinline__ void apply(const GroupRows &G, int k, T d) const {
        if (x == nullptr) return;
        const double v = x[G.rp[k]] + (double)d;
        store_h(x, G, k, v);
        if (xh) {
            const float h = (float)v;
            store_h(xh, G, k, h);
            store_h(xl, G, k, (float)(v - (double)h));
        }
    }
};

// MODE 0: y = b + K x (b may be null); MODE 1: y = x - K x
template <typename T, int MODE>
struct OpSpmv {
    using A = T;
    static constexpr int NA = 4;
    static constexpr bool kPart = false;
    struct Pre {
        T u;
    };
    const T *x, *b;
    T *y;
    static constexpr int kTile = sizeof(T) == 4 ? 1 : 0;
    __device__ __forceinline__ const T *gsrc(int) const { return x; }
    __device__ __forceinline__ void add_t(A *a, int k, T v, const T *s, int, NoSlot) const { a[k] += v * s[0]; }
    __device__ __forceinline__ NoSlot slot(const GraphP &, int) const { return NoSlot(); }
    __device__ __forceinline__ void add(A *a, int k, T v, int j, NoSlot) const { a[k] += v * __ldg(x + j); }
    __device__ __forceinline__ Pre pre(const GroupRows &G, int k) const {
        Pre p;
        p.u = MODE == 0 ? (b ? b[G.rp[k]] : T(0)) : x[G.rp[k]];
        return p;
    }
    template <int W>
    __device__ __forceinline__ static void combine_row(const A (*sh)[NA][32], int lane, int k, A *a) {
        sum_word<W, A, NA>(sh, lane, k, a);
    }
    __device__ __forceinline__ double finish_row(const GroupRows &G, int k, const A *a, const Pre &p) const {
        store_h(y, G, k, MODE == 0 ? p.u + a[k] : p.u - a[k]);
        return 0.0;
    }
};

// r = s - x + K x with FP64 x and FP64 accumulation; partial sums of r^2
template <typename T>
struct OpResid64 {
    using A = double;
    static constexpr int NA = 4;
    static constexpr bool kPart = true;
    struct Pre {
        double s, x;
    };
    const T *s;
    const double *x;
    double *r, *part;
    __device__ __forceinline__ NoSlot slot(const GraphP &, int) const { return NoSlot(); }
    __device__ __forceinline__ void add(A *a, int k, T v, int j, NoSlot) const { a[k] += (double)v * __ldg(x + j); }
    __device__ __forceinline__ Pre pre(const GroupRows &G, int k) const {
        Pre p;
        p.s = (double)s[G.row[k]];
        p.x = x[G.rp[k]];
        return p;
    }
    template <int W>
    __device__ __forceinline__ static void combine_row(const A (*sh)[NA][32], int lane, int k, A *a) {
        sum_word<W, A, NA>(sh, lane, k, a);
    }
    __device__ __forceinline__ double finish_row(const GroupRows &G, int k, const A *a, const Pre &p) const {
        const double vv = p.s - p.x + a[k];
        store_h(r, G, k, vv);
        return vv * vv;
    }
};

// Neumann sweep y = b + K x with partial sums of (y - x)^2
template <typename T>
struct OpSweepPow {
    using A = T;
    static constexpr int NA = 4;
    static constexpr bool kPart = true;
    struct Pre {
        T b, x;
    };
    const T *x, *b;
    T *y;
    double *part;
    XUpd xu;
    static constexpr int kTile = sizeof(T) == 4 ? 1 : 0;
    __device__ __forceinline__ const T *gsrc(int) const { return x; }
    __device__ __forceinline__ void add_t(A *a, int k, T v, const T *s, int, NoSlot) const { a[k] += v * s[0]; }
    __device__ __forceinline__ NoSlot slot(const GraphP &, int) const { return NoSlot(); }
    __device__ __forceinline__ void add(A *a, int k, T v, int j, NoSlot) const { a[k] += v * __ldg(x + j); }
    __device__ __forceinline__ Pre pre(const GroupRows &G, int k) const {
        Pre p;
        p.b = b[G.rp[k]];
        p.x = x[G.rp[k]];
        return p;
    }
    template <int W>
    __device__ __forceinline__ static void combine_row(const A (*sh)[NA][32], int lane, int k, A *a) {
        sum_word<W, A, NA>(sh, lane, k, a);
    }
    __device__ __forceinline__ double finish_row(const GroupRows &G, int k, const A *a, const Pre &p) const {
        const T vv = p.b + a[k];
        const T dd = vv - p.x;
        store_h(y, G, k, vv);
        xu.apply(G, k, vv);
        return (double)(dd * dd);
    }
};

// One Chebyshev step on (I - K) d = r0 (three-term form):
//   q = K p;  r <- r - p + q;  d <- d + p;  p' = c1 p + c2 r
template <typename T>
struct OpCheb {
    using A = T;
    static constexpr int NA = 4;
    static constexpr bool kPart = false;
    struct Pre {
        T p, r, d;
    };
    const T *p;
    T *r, *d, *pn;
    T c1, c2;
    XUpd xu;
    static constexpr int kTile = sizeof(T) == 4 ? 1 : 0;
    __device__ __forceinline__ const T *gsrc(int) const { return p; }
    __device__ __forceinline__ void add_t(A *a, int k, T v, const T *s, int, NoSlot) const { a[k] += v * s[0]; }
    __device__ __forceinline__ NoSlot slot(const GraphP &, int) const { return NoSlot(); }
    __device__ __forceinline__ void add(A *a, int k, T v, int j, NoSlot) const { a[k] += v * __ldg(p + j); }
    __device__ __forceinline__ Pre pre(const GroupRows &G, int k) const {
        const int ip = G.rp[k];
        Pre q;
        q.p = p[ip];
        q.r = r[ip];
        q.d = d[ip];
        return q;
    }
    template <int W>
    __device__ __forceinline__ static void combine_row(const A (*sh)[NA][32], int lane, int k, A *a) {
        sum_word<W, A, NA>(sh, lane, k, a);
    }
    __device__ __forceinline__ double finish_row(const GroupRows &G, int k, const A *a, const Pre &q) const {
        const T rr = q.r - q.p + a[k];
        store_h(r, G, k, rr);
        const T dn = q.d + q.p;
        store_h(d, G, k, dn);
        xu.apply(G, k, dn);
        store_h(pn, G, k, c1 * q.p + c2 * rr);
        return 0.0;
    }
};

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

// r = s - x + K x with K x summed in FP32 pairs (a[k]: high part, a[4 + k]: low part)
struct OpResidDS {
    using A = float;
    static constexpr int NA = 8;
    static constexpr bool kPart = true;
    struct Pre {
        double s, x;
    };
    const float *s;
    const double *x;
    const float *xh, *xl;
    double *r, *part;
    __device__ __forceinline__ NoSlot slot(const GraphP &, int) const { return NoSlot(); }
    __device__ __forceinline__ void add(A *a, int k, float v, int j, NoSlot) const {
        ds_add_prod(a[k], a[4 + k], v, __ldg(xh + j), __ldg(xl + j));
    }
    static constexpr int kTile = 2;
    __device__ __forceinline__ const float *gsrc(int i) const { return i == 0 ? xh : xl; }
    __device__ __forceinline__ void add_t(A *a, int k, float v, const float *s, int st, NoSlot) const {
        ds_add_prod(a[k], a[4 + k], v, s[0], s[st]);
    }
    __device__ __forceinline__ Pre pre(const GroupRows &G, int k) const {
        Pre p;
        p.s = (double)s[G.row[k]];
        p.x = x[G.rp[k]];
        return p;
    }
    // the W (hi, lo) partials of row k combined with FP32 two-sums
    template <int W>
    __device__ __forceinline__ static void combine_row(const A (*sh)[NA][32], int lane, int k, A *a) {
        float h = 0.f, l = 0.f;
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const float pp = sh[q][k][lane];
            const float ss = __fadd_rn(h, pp);
            const float bb = __fsub_rn(ss, h);
            l = __fadd_rn(l, __fadd_rn(__fadd_rn(__fsub_rn(h, __fsub_rn(ss, bb)), __fsub_rn(pp, bb)),
                                       sh[q][k + 4][lane]));
            h = ss;
        }
        a[k] = h;
        a[k + 4] = l;
    }
    __device__ __forceinline__ double finish_row(const GroupRows &G, int k, const A *a, const Pre &p) const {
        const double vv = p.s - p.x + ((double)a[k] + (double)a[k + 4]);
        store_h(r, G, k, vv);
        return vv * vv;
    }
};

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

// partial sums of a sweep or residual pass: one per row block (4 per group)
int sweep_blocks(const GridC &g) { return 4 * (g.nz + 1) * g.gpl; }
int resid_blocks(const GridC &g) { return sweep_blocks(g); }

bool stage_fits(int ntmax) { return ntmax > 0; }

// Warps per group (measured on GB300, plume 64 x 64 x 32, interleaved runs):
// the streamed passes run 16 consumer warps per SM; the plain passes with
// programmatic launches are fastest with 6 warps per group while all groups
// fit in one wave of resident blocks, else with the count that fills the
// last wave best.
template <typename T>
int choose_wq_t(const GridC &g) {
    if (sizeof(T) == 4 && g.stage) return 16;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms <= 0)
        return 6;
    const long long blocks = (long long)(g.nz + 1) * g.gpl;
    int best = 6;
    double best_eff = -1.0;
    const int cand[3] = {6, 8, 4};
    for (int i = 0; i < 3; ++i) {
        int w = cand[i], bps = 0;
        cudaError_t e;
        if (w == 8)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_plain<8, T, OpCheb<T>>, 32 * 8, 0);
        else if (w == 6)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_plain<6, T, OpCheb<T>>, 32 * 6, 0);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_plain<4, T, OpCheb<T>>, 32 * 4, 0);
        if (e != cudaSuccess || bps <= 0) continue;
        const double waves = (double)blocks / ((double)sms * bps);
        if (w == 6 && waves <= 1.0) {
            best = 6;
            break;
        }
        const double eff = waves / std::ceil(waves);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = w;
        }
    }
    cudaGetLastError();  // clear a failed occupancy query
    return best;
}

int choose_wq(const GridC &g, bool fp64) { return fp64 ? choose_wq_t<double>(g) : choose_wq_t<float>(g); }

template <typename T>
void launch_spmv(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, const T *b, T *y) {
    OpSpmv<T, 0> op;
    op.x = x;
    op.b = b;
    op.y = y;
    run_op(st, g, gp, val, op, 0);
}

template <typename T>
void launch_imk(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, T *y) {
    OpSpmv<T, 1> op;
    op.x = x;
    op.b = nullptr;
    op.y = y;
    run_op(st, g, gp, val, op, 0);
}

template <typename T>
void launch_sweep_pow(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *x, const T *b, T *y,
                      double *part, double *x64, float *xh, float *xl) {
    OpSweepPow<T> op;
    op.x = x;
    op.b = b;
    op.y = y;
    op.part = part;
    op.xu.x = x64;
    op.xu.xh = xh;
    op.xu.xl = xl;
    run_op(st, g, gp, val, op, 0);
}

template <typename T>
void launch_cheb(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *p, T *r, T *d, T *pn,
                 double c1, double c2, double *x64, float *xh, float *xl) {
    OpCheb<T> op;
    op.xu.x = x64;
    op.xu.xh = xh;
    op.xu.xl = xl;
    op.p = p;
    op.r = r;
    op.d = d;
    op.pn = pn;
    op.c1 = (T)c1;
    op.c2 = (T)c2;
    run_op(st, g, gp, val, op, 0);
}

// ---------------------------------------------------------------------------
// Chebyshev refinements of several scenes in one persistent launch (the
// serving loop's batches, batch.h).  Tile t of the launch is row group
// t - tile0 of the job whose tiles hold it; block b handles tiles b, b + G,
// b + 2G, ... in every step (G = gridDim.x), so the rows a block finishes are
// always its own; the gathered vector comes from other blocks and is read
// around L1.  Between steps a grid-wide barrier: every wait is bounded, and a
// barrier that gives up sets the launch's abort flag, after which every
// block skips the remaining steps and the jobs' scenes get STATUS_TIMEOUT.
constexpr long long kBarrierPolls = 1ll << 21;  // with a 256 ns sleep per poll: about a second

__device__ bool grid_barrier(BatchBarrier *b, unsigned nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *vgen = &b->gen;
        volatile int *vab = &b->abort;
        if (*vab) {
            ok = 0;
        } else {
            const unsigned g0 = *vgen;  // read before arriving: the last arrival changes it
            __threadfence();
            if (atomicAdd(&b->count, 1u) + 1u == nblocks) {
                atomicExch(&b->count, 0u);
                __threadfence();
                atomicAdd(&b->gen, 1u);
            } else {
                for (long long i = 0; *vgen == g0; ++i) {
                    if (*vab) {
                        ok = 0;
                        break;
                    }
                    if (i >= kBarrierPolls) {
                        atomicExch(&b->abort, 1);
                        atomicOr(&b->status, STATUS_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(256);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

int batch_tiles(const GridC &g) { return (g.nz + 1) * g.gpl; }

template <int W>
__global__ void __launch_bounds__(32 * W) k_cheb_batch(const ChebJob *__restrict__ jobs, int njobs, int ntiles,
                                                      int max_steps, BatchBarrier *bar) {
    __shared__ float sh[W][4][32];
    extern __shared__ float tile[];
    __shared__ int s_lay[kTileLayers];
    __shared__ ChebJob sj;
    __shared__ int s_tile0[kChebMaxJobs + 1];
    for (int i = threadIdx.x; i <= njobs; i += blockDim.x) s_tile0[i] = i < njobs ? jobs[i].tile0 : ntiles;
    __syncthreads();
    int cur = -1;
    for (int step = 0; step < max_steps; ++step) {
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int j = 0;
            while (j + 1 < njobs && s_tile0[j + 1] <= t) ++j;
            if (j != cur) {  // the job's constants into shared memory
                __syncthreads();
                const int4 *src = reinterpret_cast<const int4 *>(jobs + j);
                int4 *dst = reinterpret_cast<int4 *>(&sj);
                for (int k = threadIdx.x; k < (int)(sizeof(ChebJob) / 16); k += blockDim.x) dst[k] = src[k];
                __syncthreads();
                cur = j;
            }
            if (step >= sj.nsteps) continue;
            OpCheb<float> op;
            op.p = sj.p[step & 1];
            op.pn = sj.p[(step + 1) & 1];
            op.r = sj.r;
            op.d = sj.d;
            op.c1 = sj.c1[step];
            op.c2 = sj.c2[step];
            if (step == sj.nsteps - 1) {
                op.xu.x = sj.x64;
                op.xu.xh = sj.xh;
                op.xu.xl = sj.xl;
            }
            __syncthreads();
            tile_group<W, OpCheb<float>, false, true>(sj.g, sj.gp, sj.val, op, t - sj.tile0, sh, tile, s_lay);
        }
        if (!grid_barrier(bar, gridDim.x)) break;
    }
    __syncthreads();
    // a barrier that gave up: every job's scene learns it at its next read-back
    if (threadIdx.x == 0 && *(volatile int *)&bar->abort)
        for (int j = blockIdx.x; j < njobs; j += gridDim.x) atomicOr(jobs[j].gp.status, STATUS_TIMEOUT);
}

bool batch_eligible(const GridC &g, int nsteps) {
    return nsteps >= 1 && nsteps <= kChebMaxSteps && !g.stage && g.tl > 0 && batch_tiles(g) <= kBatchMaxTiles &&
           (size_t)kTileLayers * g.tl * sizeof(float) <= (size_t)kTileMaxBytes &&
           (g.wq == 4 || g.wq == 6 || g.wq == 8);
}

template <int W>
static cudaError_t launch_cheb_batch_w(cudaStream_t st, const ChebJob *d_jobs, const ChebJob *h_jobs, int njobs,
                                       BatchBarrier *bar, int share) {
    int ntiles = 0, max_steps = 0, tl = 0;
    for (int j = 0; j < njobs; ++j) {
        ntiles += batch_tiles(h_jobs[j].g);
        max_steps = max(max_steps, h_jobs[j].nsteps);
        tl = max(tl, h_jobs[j].g.tl);
    }
    const size_t smem = (size_t)kTileLayers * tl * sizeof(float);
    int dev = 0, nsm = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cheb_batch<W>, 32 * W, smem);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const int grid = min(ntiles, max(1, per * nsm / max(1, share)));
    void *args[] = {(void *)&d_jobs, (void *)&njobs, (void *)&ntiles, (void *)&max_steps, (void *)&bar};
    return cudaLaunchCooperativeKernel((const void *)k_cheb_batch<W>, dim3(grid), dim3(32 * W), args, smem, st);
}

cudaError_t launch_cheb_batch(cudaStream_t st, const ChebJob *d_jobs, const ChebJob *h_jobs, int njobs, int W,
                              BatchBarrier *bar, int share) {
    if (njobs < 1 || njobs > kChebMaxJobs) return cudaErrorInvalidValue;
    if (W == 4) return launch_cheb_batch_w<4>(st, d_jobs, h_jobs, njobs, bar, share);
    if (W == 6) return launch_cheb_batch_w<6>(st, d_jobs, h_jobs, njobs, bar, share);
    if (W == 8) return launch_cheb_batch_w<8>(st, d_jobs, h_jobs, njobs, bar, share);
    return cudaErrorInvalidValue;
}

// the self-test: every block meets one barrier that expects `expect` arrivals
__global__ void k_barrier_test(BatchBarrier *bar, unsigned expect) { grid_barrier(bar, expect); }

int batch_barrier_selftest(cudaStream_t st, int blocks, int arrive) {
    BatchBarrier *bar = nullptr;
    if (cudaMalloc((void **)&bar, sizeof(BatchBarrier)) != cudaSuccess) return -1;
    int result = -1;
    BatchBarrier h{};
    if (cudaMemsetAsync(bar, 0, sizeof(BatchBarrier), st) == cudaSuccess) {
        unsigned expect = (unsigned)blocks + (arrive ? 0u : 1u);
        void *args[] = {(void *)&bar, (void *)&expect};
        if (cudaLaunchCooperativeKernel((const void *)k_barrier_test, dim3(blocks), dim3(32), args, 0, st) ==
                cudaSuccess &&
            cudaMemcpyAsync(&h, bar, sizeof(h), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess)
            result = h.status & STATUS_TIMEOUT;
    }
    cudaFree(bar);
    return result;
}

bool resid_ds_ok(const GridC &g) { return true; }

void launch_resid_ds(cudaStream_t st, const GridC &g, const GraphP &gp, const float *val, const float *s,
                     const double *x, const float *xh, const float *xl, double *r, double *part, int nblk) {
    (void)nblk;
    OpResidDS op;
    op.s = s;
    op.x = x;
    op.xh = xh;
    op.xl = xl;
    op.r = r;
    op.part = part;
    run_op(st, g, gp, val, op, 0);
}

template <typename T>
void launch_update_x(cudaStream_t st, int n, const T *d, double *x, float *xh, float *xl) {
    k_update_x<T><<<(n + 255) / 256, 256, 0, st>>>(n, d, x, xh, xl);
}

template <typename T>
void launch_resid64(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const T *s, const double *x,
                    double *r, double *part, int nblk) {
    (void)nblk;
    OpResid64<T> op;
    op.s = s;
    op.x = x;
    op.r = r;
    op.part = part;
    run_op(st, g, gp, val, op, 0);
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

// ---------------------------------------------------------------------------
// Reductions

// Dot products over the nodes of haloed vectors (each node once, halo
// copies skipped): warp per line of nx nodes, lines strided over the grid.
template <typename A, typename B>
__global__ void k_dots(GridC g, const A *__restrict__ V, size_t ldv, int ncol, const B *__restrict__ y,
                       double *__restrict__ part) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5), nw = gridDim.x * wpb;
    const int nlines = (g.nz + 1) * g.ny;
    for (int k = 0; k < ncol; ++k) {
        const A *v = V + (size_t)k * ldv;
        double acc = 0.0;
        for (int l = gw; l < nlines; l += nw) {
            const int z = l / g.ny, yy = l - z * g.ny;
            const long long base = halo_pos(g, 0, yy, z);
            for (int x = lane; x < g.nx; x += 32) acc += (double)v[base + x] * (double)y[base + x];
        }
        double b = block_sum(acc);
        if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = b;
    }
}

// one block per column; fixed strided partial sums then a fixed-order tree
// Column k of the block partials part[k][nblk] summed into out[k] by one
// block of kFinThreads threads: each thread adds its strided share with four
// loads in flight at a time (one memory round trip per four values instead
// of one per value), then the warps' fixed butterflies and warp 0 over the
// warps' sums.  The order depends on nblk only, so the sum is deterministic.
constexpr int kFinThreads = 1024;
__global__ void __launch_bounds__(kFinThreads) k_finalize(const double *__restrict__ part, int nblk, int ncol,
                                                         double *__restrict__ out) {
    __shared__ double sh[32];
    const int k = blockIdx.x;
    const double *p = part + (size_t)k * nblk;
    double s = 0.0;
    int b = threadIdx.x;
    for (; b + 3 * kFinThreads < nblk; b += 4 * kFinThreads) {
        const double a0 = p[b], a1 = p[b + kFinThreads], a2 = p[b + 2 * kFinThreads], a3 = p[b + 3 * kFinThreads];
        s += (a0 + a1) + (a2 + a3);
    }
    for (; b < nblk; b += kFinThreads) s += p[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = s;
    __syncthreads();
    if (w == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) out[k] = t;
    }
    (void)ncol;
}

int dot_blocks(const GridC &g) {
    long long b = ((long long)(g.nz + 1) * g.ny + 7) / 8;
    if (b > 296) b = 296;
    if (b < 1) b = 1;
    return (int)b;
}

// The same dot products for FP32 vectors without FP64 arithmetic in the
// pass (FP64 runs at a small fraction of the FP32 rate on this GPU): each
// product and each thread's running sum is kept in FP32-pair arithmetic
// (ds_add_prod, about 48 significant bits), kDotCols columns per pass over
// y; the pairs enter the FP64 block and grid sums only at the end.
constexpr int kDotCols = 8;
// blocks per SM (measured on the 128 x 128 x 40 cloud: 4 beats 2; a flat
// element decomposition at 4 or 8 blocks per SM was slower than warps per line)
constexpr int kDotBlocksPerSM = 4;
// (hi, lo) += (h2, l2) for FP32 pairs, with Knuth's two-sum on the high parts
__device__ __forceinline__ void ds_add_pair(float &hi, float &lo, float h2, float l2) {
    const float s = __fadd_rn(hi, h2);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, l2));
}
__global__ void __launch_bounds__(256) k_dots_ds(GridC g, const float *__restrict__ V, size_t ldv, int ncol,
                                                 const float *__restrict__ y, double *__restrict__ part) {
    __shared__ double red[kDotCols][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * 8 + wid, nw = gridDim.x * 8;
    const int nlines = (g.nz + 1) * g.ny;
    for (int c0 = 0; c0 < ncol; c0 += kDotCols) {
        float hi[kDotCols], lo[kDotCols];
#pragma unroll
        for (int c = 0; c < kDotCols; ++c) hi[c] = lo[c] = 0.f;
        for (int l = gw; l < nlines; l += nw) {
            const int z = l / g.ny, yy = l - z * g.ny;
            const long long base = halo_pos(g, 0, yy, z);
#pragma unroll 4
            for (int x = lane; x < g.nx; x += 32) {
                const float yv = y[base + x];
#pragma unroll
                for (int c = 0; c < kDotCols; ++c)
                    if (c0 + c < ncol) ds_add_prod(hi[c], lo[c], V[(size_t)(c0 + c) * ldv + base + x], yv, 0.f);
            }
        }
        // warp sums in FP32-pair arithmetic; FP64 only for the warps' results
#pragma unroll
        for (int c = 0; c < kDotCols; ++c) {
            float h = hi[c], q = lo[c];
            for (int o = 16; o > 0; o >>= 1)
                ds_add_pair(h, q, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, q, o));
            if (lane == 0) red[c][wid] = (double)h + (double)q;
        }
        __syncthreads();
        if (threadIdx.x < kDotCols && c0 + (int)threadIdx.x < ncol) {
            double t = 0.0;
            for (int q = 0; q < 8; ++q) t += red[threadIdx.x][q];
            part[(size_t)(c0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

int dot_blocks_ds() {
    static int n = 0;
    if (!n) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        n = std::max(1, sms) * kDotBlocksPerSM;
    }
    return n;
}

template <typename A, typename B>
void launch_dots(cudaStream_t st, const GridC &g, const A *V, size_t ldv, int ncol, const B *y, double *part,
                 int nblk, double *out) {
    if constexpr (sizeof(A) == 4 && sizeof(B) == 4) {
        const int nb = std::min(dot_blocks_ds(), std::max(1, (g.nz + 1) * g.ny / 8));
        k_dots_ds<<<nb, 256, 0, st>>>(g, (const float *)V, ldv, ncol, (const float *)y, part);
        k_finalize<<<ncol, kFinThreads, 0, st>>>(part, nb, ncol, out);
        return;
    }
    k_dots<A, B><<<nblk, 256, 0, st>>>(g, V, ldv, ncol, y, part);
    k_finalize<<<ncol, kFinThreads, 0, st>>>(part, nblk, ncol, out);
}

template <typename T>
void launch_sumsq(cudaStream_t st, const GridC &g, const T *x, double *part, int nblk, double *out) {
    launch_dots<T, T>(st, g, x, 0, 1, x, part, nblk, out);
}

// haloed dst <- node-ordered src (every halo copy written)
template <typename T, typename U>
__global__ void k_to_halo(GridC g, const T *__restrict__ src, U *__restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_nodes) return;
    const int z = i / g.nxy, r = i - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    const long long p = halo_pos(g, x, y, z);
    const int ax = x < g.H ? g.nx : (x >= g.nx - g.H ? -g.nx : 0);
    const int ay = y < g.H ? g.ny * g.nxp : (y >= g.ny - g.H ? -g.ny * g.nxp : 0);
    const U v = (U)src[i];
    dst[p] = v;
    if (ax) dst[p + ax] = v;
    if (ay) {
        dst[p + ay] = v;
        if (ax) dst[p + ax + ay] = v;
    }
}

// node-ordered dst <- haloed src
template <typename U>
__global__ void k_from_halo(GridC g, const U *__restrict__ src, U *__restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_nodes) return;
    const int z = i / g.nxy, r = i - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    dst[i] = src[halo_pos(g, x, y, z)];
}

template <typename T, typename U>
void launch_to_halo(cudaStream_t st, const GridC &g, const T *src, U *dst) {
    k_to_halo<T, U><<<(g.n_nodes + 255) / 256, 256, 0, st>>>(g, src, dst);
}

template <typename U>
void launch_from_halo(cudaStream_t st, const GridC &g, const U *src, U *dst) {
    k_from_halo<U><<<(g.n_nodes + 255) / 256, 256, 0, st>>>(g, src, dst);
}

void launch_finalize2(cudaStream_t st, const double *part, int nblk, double *out) {
    k_finalize<<<2, kFinThreads, 0, st>>>(part, nblk, 2, out);
}

void launch_finalize(cudaStream_t st, const double *part, int nblk, double *out) {
    k_finalize<<<1, kFinThreads, 0, st>>>(part, nblk, 1, out);
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
__global__ void k_add(int n, T *a, const T *b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += b[i];
}
template <typename T>
__global__ void k_cheb_start(int n, const double *__restrict__ r64, double alpha, T *__restrict__ b,
                             T *__restrict__ d, T *__restrict__ p) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T v = (T)r64[i];
    b[i] = v;
    d[i] = T(0);
    p[i] = (T)(alpha * (double)v);
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

// w += sign sum_j h_j V_j for FP32 vectors in FP32-pair arithmetic: the
// coefficients are split once per block into (high, low) FP32 pairs, and
// each element's sum is carried as a pair and rounded to FP32 at the end
constexpr int kGupdateMaxK = 64;
template <bool kNorm>
__global__ void __launch_bounds__(256) k_gupdate_ds(GridC g, int n, float *__restrict__ w, const float *__restrict__ V,
                                                    size_t ldv, int k, const double *__restrict__ h, double sign,
                                                    double *__restrict__ part) {
    __shared__ float hh[kGupdateMaxK], hl[kGupdateMaxK];
    __shared__ double red[8];
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double c = sign * h[j];
        const float a = (float)c;
        hh[j] = a;
        hl[j] = (float)(c - (double)a);
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float r = 0.f;
    if (i < n) {
        float hi = w[i], lo = 0.f;
#pragma unroll 4
        for (int j = 0; j < k; ++j) ds_add_prod(hi, lo, V[(size_t)j * ldv + i], hh[j], hl[j]);
        r = __fadd_rn(hi, lo);
        w[i] = r;
    }
    if constexpr (kNorm) {
        // ||w||^2 over the interior (halo copies excluded), as FP32 pairs per
        // warp and FP64 per block: part[blockIdx.x]
        float sh = 0.f, sl = 0.f;
        if (i < n) {
            const int rem = i % g.lp, yy = rem / g.nxp, xx = rem - yy * g.nxp;
            if (xx >= g.H && xx < g.nx + g.H && yy >= g.H && yy < g.ny + g.H) ds_add_prod(sh, sl, r, r, 0.f);
        }
        for (int o = 16; o > 0; o >>= 1)
            ds_add_pair(sh, sl, __shfl_xor_sync(0xffffffffu, sh, o), __shfl_xor_sync(0xffffffffu, sl, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)sh + (double)sl;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
            part[blockIdx.x] = t;
        }
    }
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
void launch_add(cudaStream_t st, int n, T *a, const T *b) {
    k_add<T><<<(n + 255) / 256, 256, 0, st>>>(n, a, b);
}
template <typename T>
void launch_cheb_start(cudaStream_t st, int n, const double *r64, double alpha, T *b, T *d, T *p) {
    k_cheb_start<T><<<(n + 255) / 256, 256, 0, st>>>(n, r64, alpha, b, d, p);
}
template <typename T>
void launch_gmres_update(cudaStream_t st, int n, T *w, const T *V, size_t ldv, int k, const double *h) {
    if constexpr (sizeof(T) == 4) {
        k_gupdate_ds<false><<<(n + 255) / 256, 256, 0, st>>>(GridC(), n, (float *)w, (const float *)V, ldv, k, h,
                                                               -1.0, nullptr);
        return;
    }
    k_gupdate<T><<<(n + 255) / 256, 256, 0, st>>>(n, w, V, ldv, k, h, -1.0);
}
// w -= V h, then ||w||^2 (interior) into *out; part: scratch partial sums
template <typename T>
void launch_gmres_update_norm(cudaStream_t st, const GridC &g, int n, T *w, const T *V, size_t ldv, int k,
                              const double *h, double *part, int nblk, double *out) {
    if constexpr (sizeof(T) == 4) {
        const int nb = (n + 255) / 256;
        k_gupdate_ds<true><<<nb, 256, 0, st>>>(g, n, (float *)w, (const float *)V, ldv, k, h, -1.0, part);
        k_finalize<<<1, kFinThreads, 0, st>>>(part, nb, 1, out);
        return;
    }
    launch_gmres_update<T>(st, n, w, V, ldv, k, h);
    launch_sumsq<T>(st, g, w, part, nblk, out);
}

template <typename T>
void launch_combine(cudaStream_t st, int n, T *x, const T *V, size_t ldv, int k, const double *y) {
    if constexpr (sizeof(T) == 4) {
        k_gupdate_ds<false><<<(n + 255) / 256, 256, 0, st>>>(GridC(), n, (float *)x, (const float *)V, ldv, k, y, 1.0,
                                                               nullptr);
        return;
    }
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
    template void launch_dots<T, T>(cudaStream_t, const GridC &, const T *, size_t, int, const T *, double *, int,  \
                                    double *);                                                                      \
    template void launch_sumsq<T>(cudaStream_t, const GridC &, const T *, double *, int, double *);                 \
    template void launch_to_halo<T, double>(cudaStream_t, const GridC &, const T *, double *);                      \
    template void launch_from_halo<T>(cudaStream_t, const GridC &, const T *, T *);                                 \
    template void launch_axpy_to64<T>(cudaStream_t, int, const T *, double *);                                      \
    template void launch_scale<T>(cudaStream_t, int, const T *, double, T *);                                       \
    template void launch_cheb_start<T>(cudaStream_t, int, const double *, double, T *, T *, T *);                  \
    template void launch_add<T>(cudaStream_t, int, T *, const T *);                                                \
    template void launch_gmres_update<T>(cudaStream_t, int, T *, const T *, size_t, int, const double *);           \
    template void launch_gmres_update_norm<T>(cudaStream_t, const GridC &, int, T *, const T *, size_t, int,       \
                                              const double *, double *, int, double *);                          \
    template void launch_combine<T>(cudaStream_t, int, T *, const T *, size_t, int, const double *);            \
    template void launch_axpby<T>(cudaStream_t, int, double, const T *, double, const T *, T *);                   \
    template void launch_update_x<T>(cudaStream_t, int, const T *, double *, float *, float *);                   \
    template void launch_sweep_pow<T>(cudaStream_t, const GridC &, const GraphP &, const T *, const T *,          \
                                      const T *, T *, double *, double *, float *, float *);                    \
    template void launch_cheb<T>(cudaStream_t, const GridC &, const GraphP &, const T *, const T *, T *, T *,     \
                                 T *, double, double, double *, float *, float *);
INST(float)
INST(double)
#undef INST
template void launch_to_halo<float, float>(cudaStream_t, const GridC &, const float *, float *);
template void launch_convert<double, float>(cudaStream_t, int, const double *, float *);
template void launch_convert<float, double>(cudaStream_t, int, const float *, double *);
template void launch_convert<double, double>(cudaStream_t, int, const double *, double *);
template void launch_convert<float, float>(cudaStream_t, int, const float *, float *);

}  // namespace tk
