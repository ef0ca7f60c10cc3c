// Row groups of the solver kernels and the bulk-copy pipeline that streams
// the matrix values of FP32 scenes through shared memory.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "kern.h"

namespace tk {

// ---- Row groups.  Group gi = z * gpl + q is the q-th run of kGroup = 128
// rows of layer z; lane l of a warp owns rows q * 128 + l + 32 k (k = 0..3).
// The values of one group are a contiguous run of nt * 128 elements (slot
// major: slot t, row r at vb + t * 128 + r), so each value load, gather and
// store of a warp covers one contiguous 128-byte line.
struct GroupRows {
    int z, nt, t0;
    long long vb;  // value index of slot 0 of this group
    int row[4];    // node index of each owned row (-1: past the end of the layer)
    int rp[4];     // haloed position of the row (rows past the end: a node of the layer)
    int ax[4];     // offset of the row's halo copy in x (0: none)
    int ay[4];     // offset of the row's halo copy in y (0: none)
};

__device__ __forceinline__ GroupRows group_rows(const GridC &g, const GraphP &gp, int gi) {
    GroupRows G;
    const int lane = threadIdx.x & 31;
    G.z = gi / g.gpl;
    const int q = gi - G.z * g.gpl;
    G.t0 = __ldg(gp.tstart + G.z);
    G.nt = __ldg(gp.tstart + G.z + 1) - G.t0;
    G.vb = __ldg(gp.voff + G.z) + (long long)q * G.nt * kGroup;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = q * kGroup + lane + 32 * k;
        const bool ok = r < g.nxy;
        const int rr = ok ? r : 0;
        const int y = rr / g.nx, x = rr - y * g.nx;
        G.row[k] = ok ? G.z * g.nxy + r : -1;
        G.rp[k] = (int)halo_pos(g, x, y, G.z);
        G.ax[k] = x < g.H ? g.nx : (x >= g.nx - g.H ? -g.nx : 0);
        G.ay[k] = y < g.H ? g.ny * g.nxp : (y >= g.ny - g.H ? -g.ny * g.nxp : 0);
    }
    return G;
}

// store a row's value at its haloed position and at every halo copy of it
template <typename T>
__device__ __forceinline__ void store_h(T *v, const GroupRows &G, int k, T val) {
    const int p = G.rp[k];
    v[p] = val;
    if (G.ax[k]) v[p + G.ax[k]] = val;
    if (G.ay[k]) {
        v[p + G.ay[k]] = val;
        if (G.ax[k]) v[p + G.ax[k] + G.ay[k]] = val;
    }
}

// iterations of the slot loop kept in flight per warp (plain driver)
#ifndef TK_SWEEP_UNROLL
#define TK_SWEEP_UNROLL 4
#endif
constexpr int kSweepUnroll = TK_SWEEP_UNROLL;

// word m of the accumulators summed over the W warps' partials in order
template <int W, typename A, int NA>
__device__ __forceinline__ void sum_word(const A (*sh)[NA][32], int lane, int m, A *a) {
    A t = A(0);
#pragma unroll
    for (int q = 0; q < W; ++q) t += sh[q][m][lane];
    a[m] = t;
}

// warp sum of one double, written by lane 0
__device__ __forceinline__ void warp_partial(double v, double *part, int idx) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[idx] = v;
}

// warp k (< 4) finishes row block k of the group: combine, update, partial sum
template <int W, class Op>
__device__ __forceinline__ void finish_rows(const Op &op, const typename Op::A (*sh)[Op::NA][32], const GroupRows &G,
                                            const typename Op::Pre &pre, int gi) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= 4) return;
    typename Op::A a[Op::NA];
    Op::template combine_row<W>(sh, lane, w, a);
    const double v = G.row[w] >= 0 ? op.finish_row(G, w, a, pre) : 0.0;
    if constexpr (Op::kPart) warp_partial(v, op.part, 4 * gi + w);
}

// epilogue inputs of row block w (< 4) of the group
template <class Op>
__device__ __forceinline__ typename Op::Pre load_pre(const Op &op, const GroupRows &G) {
    const int w = threadIdx.x >> 5;
    typename Op::Pre p{};
    if (w < 4 && G.row[w] >= 0) p = op.pre(G, w);
    return p;
}

// no per-slot constants
struct NoSlot {};

// ---- Bulk-copy pipeline (FP32 values).  One persistent block per SM
// streams one contiguous run of groups [g0, g1) -- the groups' values are
// stored back to back, so the run is one contiguous byte range -- through a
// ring of kPipeStages shared-memory stages.  Its last warp is the producer:
// one lane copies the range in chunks of kPipeRows slot rows (a slot row is
// the 128 values of one slot of one group, 512 bytes in FP32), 32 KiB per
// cp.async.bulk, each chunk's arrival counted in bytes on the stage's "full"
// mbarrier.  Chunks ignore group boundaries.  The W consumer warps walk the
// same chunks, keep a cursor (group, slot) over the run, add slot t of the
// current group in warp t mod W (as the plain driver does, so both give the
// same bits), finish each group when its last slot has been added, and
// release each stage on its "empty" mbarrier (one arrival per warp).
// Large chunks matter: a block sustains roughly one bulk copy per few
// hundred nanoseconds, so small copies cap the stream well below HBM speed.
//
// Every wait is bounded: a wait that gives up after kWaitTries polls sets
// STATUS_TIMEOUT in the scene status and the block's abort flag, after which
// the block's remaining waits return at once; the block then still runs to
// the end without depending on the staged data for any address or branch,
// and before it exits waits (bounded, regardless of the flag) for copies it
// may still have in flight.
constexpr int kPipeRows = 64;                          // slot rows per chunk
constexpr int kPipeStageFloats = kPipeRows * kGroup;   // 32 KiB
constexpr int kWaitTries = 1 << 18;                    // polls of one barrier: about 1 s on GB300, where a
                                                       // poll that finds the phase incomplete suspends the
                                                       // thread for about 3.7 us (2^22 polls measured 15.7 s)

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_poll(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// one arrival that also announces `bytes` of transfer, then the bulk copy
// global -> shared that completes them
__device__ __forceinline__ void bulk_load(unsigned bar, void *dst, const void *src, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// bounded wait for the phase of the given parity; false after giving up
static __device__ __noinline__ bool pipe_wait(unsigned bar, unsigned parity, int *abort_flag, int *status,
                                              bool honour_abort) {
    for (int i = 0; i < kWaitTries; ++i) {
        if (mbar_poll(bar, parity)) return true;
        if (honour_abort && *(volatile int *)abort_flag) return false;
    }
    *(volatile int *)abort_flag = 1;
    atomicOr(status, STATUS_TIMEOUT);
    return false;
}

__device__ __forceinline__ void consumer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// shared memory of a pipelined launch: the ring of as many stages (up to 6)
// as fit beside two buffers of the consumers' partial sums (A: accumulator
// type, NA words per lane)
template <int W, typename A, int NA>
__host__ __device__ constexpr size_t pipe_cb_bytes() {
    return 2 * (size_t)W * NA * 32 * sizeof(A);
}
#ifndef TK_PIPE_MAX_STAGES
#define TK_PIPE_MAX_STAGES 4
#endif
template <int W, typename A, int NA>
__host__ __device__ constexpr int pipe_stages() {
    return (int)((220 * 1024 - pipe_cb_bytes<W, A, NA>()) / (kPipeStageFloats * sizeof(float))) < TK_PIPE_MAX_STAGES
               ? (int)((220 * 1024 - pipe_cb_bytes<W, A, NA>()) / (kPipeStageFloats * sizeof(float)))
               : TK_PIPE_MAX_STAGES;
}
template <int W, typename A, int NA>
__host__ __device__ constexpr size_t pipe_smem_bytes() {
    return (size_t)pipe_stages<W, A, NA>() * kPipeStageFloats * sizeof(float) + pipe_cb_bytes<W, A, NA>();
}

// The pipelined driver over the groups of pass kind `kind` (the Op
// interface is described with the ops).
template <int W, class Op>
__global__ void __launch_bounds__(32 * (W + 1), 1) k_pipe(GridC g, GraphP gp, const float *__restrict__ val, Op op,
                                                          int kind) {
    using A = typename Op::A;
    constexpr int NA = Op::NA;
    constexpr int kPipeStages = pipe_stages<W, A, NA>();
    static_assert(kPipeStages >= 2, "ring too small");
    extern __shared__ __align__(128) unsigned char dyn[];
    float *ring = (float *)dyn;
    A(*cb)[W][NA][32] = (A(*)[W][NA][32])(dyn + (size_t)kPipeStages * kPipeStageFloats * sizeof(float));
    __shared__ __align__(8) unsigned long long full[kPipeStages], empty[kPipeStages];
    __shared__ int abort_flag;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this block's run of groups (an equal share of the value stream)
    const int g0 = __ldg(gp.run_g[kind] + blockIdx.x), g1 = __ldg(gp.run_g[kind] + blockIdx.x + 1);
    const long long v0 = __ldg(gp.run_v[kind] + blockIdx.x), v1 = __ldg(gp.run_v[kind] + blockIdx.x + 1);
    const int nchunks = (int)((v1 - v0 + kPipeStageFloats - 1) / kPipeStageFloats);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kPipeStages; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), W);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (w == W) {  // producer
        if (lane == 0) {
            for (int i = 0; i < nchunks; ++i) {
                const int s = i % kPipeStages;
                if (i >= kPipeStages)
                    pipe_wait(smem_addr(&empty[s]), (unsigned)((i / kPipeStages - 1) & 1), &abort_flag, gp.status,
                              true);
                const long long off = v0 + (long long)i * kPipeStageFloats;
                const long long n = v1 - off < kPipeStageFloats ? v1 - off : kPipeStageFloats;
                bulk_load(smem_addr(&full[s]), ring + (size_t)s * kPipeStageFloats, val + off,
                          (unsigned)(n * sizeof(float)));
            }
        }
        return;
    }
    // consumers: cursor (gi, t) over the run
    int gi = g0, t = 0, gl = 0;
    GroupRows G;
    typename Op::Pre pre{};
    if (gi < g1) {
        G = group_rows(g, gp, gi);
        pre = load_pre(op, G);
    }
    A a[NA];
#pragma unroll
    for (int m = 0; m < NA; ++m) a[m] = A(0);
    // finish the current group (all warps), then move the cursor to the next
    auto end_group = [&]() {
#pragma unroll
        for (int m = 0; m < NA; ++m) cb[gl & 1][w][m][lane] = a[m];
        consumer_sync(32 * W);
        finish_rows<W>(op, cb[gl & 1], G, pre, gi);
#pragma unroll
        for (int m = 0; m < NA; ++m) a[m] = A(0);
        ++gl;
        ++gi;
        t = 0;
        if (gi < g1) {
            G = group_rows(g, gp, gi);
            pre = load_pre(op, G);
        }
    };
    while (gi < g1 && G.nt == 0) end_group();
    for (int i = 0; i < nchunks; ++i) {
        const int s = i % kPipeStages;
        pipe_wait(smem_addr(&full[s]), (unsigned)((i / kPipeStages) & 1), &abort_flag, gp.status, true);
        const long long off = v0 + (long long)i * kPipeStageFloats;
        const int rows = (int)((v1 - off < kPipeStageFloats ? v1 - off : kPipeStageFloats) / kGroup);
        const float *st = ring + (size_t)s * kPipeStageFloats + 4 * lane;
        int u = 0;  // slot rows of this chunk consumed
        while (u < rows) {
            const int seg = min(rows - u, G.nt - t);  // rows of the current group in this chunk
            // slots t .. t + seg - 1 sit at rows u .. u + seg - 1; this warp adds tt = w (mod W)
            int tt = t + ((w - t % W) + W) % W;
#pragma unroll 4
            for (; tt < t + seg; tt += W) {
                const int fp = __ldg(gp.tflat + G.t0 + tt);
                const auto si = op.slot(gp, G.t0 + tt);
                const float4 vq = *reinterpret_cast<const float4 *>(st + (size_t)(u + tt - t) * kGroup);
                const float vt[4] = {vq.x, vq.y, vq.z, vq.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) op.add(a, k, vt[k], G.rp[k] + fp, si);
            }
            u += seg;
            t += seg;
            if (t == G.nt) {
                end_group();
                while (gi < g1 && G.nt == 0) end_group();
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[s]));
    }
    // nothing of this block may still be landing when it exits
    if (threadIdx.x == 0 && *(volatile int *)&abort_flag) {
        for (int s = 0; s < kPipeStages && s < nchunks; ++s) {
            const int last = s + kPipeStages * ((nchunks - 1 - s) / kPipeStages);
            pipe_wait(smem_addr(&full[s]), (unsigned)((last / kPipeStages) & 1), &abort_flag, gp.status, false);
        }
    }
}

// The values of the four rows a lane owns in one slot row (adjacent, aligned:
// 16 bytes in FP32, 32 bytes in FP64), read once per pass.  Measured on GB300
// the plain read-only load is fastest; the L1 no-allocate and evict-first
// forms (TK_STREAM_LOAD 1, 2) are kept for experiments.
#ifndef TK_STREAM_LOAD
#define TK_STREAM_LOAD 0
#endif
#if TK_STREAM_LOAD == 1
#define TK_STREAM_QUAL "ld.global.nc.L1::no_allocate"
#elif TK_STREAM_LOAD == 2
#define TK_STREAM_QUAL "ld.global.nc.L1::evict_first"
#endif
__device__ __forceinline__ void ld_quad(const float *p, float (&v)[4]) {
#if TK_STREAM_LOAD == 0
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
#else
    asm(TK_STREAM_QUAL ".v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p));
#endif
}
__device__ __forceinline__ void ld_quad(const double *p, double (&v)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}
__device__ __forceinline__ void st_quad(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st_quad(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
// the same with the streaming (evict-first) cache hint: values written once
// and read only by later passes
__device__ __forceinline__ void st_quad_cs(float *p, const float (&v)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void st_quad_cs(double *p, const double (&v)[4]) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
    __stcs(reinterpret_cast<double2 *>(p) + 1, make_double2(v[2], v[3]));
}

// Programmatic dependent launch: a pass may be launched while the previous
// pass on the stream is still running.  Everything it reads before
// pdl_wait() (graph structure, the values of K) was written by earlier,
// completed work; pdl_wait() returns once the previous pass has completed
// and its writes are visible (a hardware wait, no polling).  pdl_trigger()
// lets the next pass launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

#ifndef TK_PDL_PEEL
#define TK_PDL_PEEL 1
#endif

// The plain driver over groups [0, gridDim.x): block gi = group gi, W warps,
// values read from global memory.  The values of each warp's first two slots
// are requested before waiting for the previous pass.
template <int W, typename T, class Op>
__global__ void __launch_bounds__(32 * W) k_plain(GridC g, GraphP gp, const T *__restrict__ val, Op op) {
    using A = typename Op::A;
    constexpr int NA = Op::NA;
    __shared__ A sh[W][NA][32];
    pdl_trigger();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const GroupRows G = group_rows(g, gp, blockIdx.x);
    const T *v = val + G.vb + 4 * lane;
    A a[NA];
#pragma unroll
    for (int m = 0; m < NA; ++m) a[m] = A(0);
#if TK_PDL_PEEL
    // the values of the warp's first two slots are requested before waiting
    T v0[4] = {T(0), T(0), T(0), T(0)}, v1[4] = {T(0), T(0), T(0), T(0)};
    const int tA = w, tB = w + W;
    if (tA < G.nt) ld_quad(v + (size_t)tA * kGroup, v0);
    if (tB < G.nt) ld_quad(v + (size_t)tB * kGroup, v1);
    pdl_wait();
    const typename Op::Pre pre = load_pre(op, G);
    if (tA < G.nt) {
        const int fp = __ldg(gp.tflat + G.t0 + tA);
        const auto si = op.slot(gp, G.t0 + tA);
#pragma unroll
        for (int k = 0; k < 4; ++k) op.add(a, k, v0[k], G.rp[k] + fp, si);
    }
    if (tB < G.nt) {
        const int fp = __ldg(gp.tflat + G.t0 + tB);
        const auto si = op.slot(gp, G.t0 + tB);
#pragma unroll
        for (int k = 0; k < 4; ++k) op.add(a, k, v1[k], G.rp[k] + fp, si);
    }
    const int tfirst = w + 2 * W;
#else
    pdl_wait();
    const typename Op::Pre pre = load_pre(op, G);
    const int tfirst = w;
#endif
#pragma unroll kSweepUnroll
    for (int t = tfirst; t < G.nt; t += W) {
        const int fp = __ldg(gp.tflat + G.t0 + t);
        const auto si = op.slot(gp, G.t0 + t);
        T q[4];
        ld_quad(v + (size_t)t * kGroup, q);
#pragma unroll
        for (int k = 0; k < 4; ++k) op.add(a, k, q[k], G.rp[k] + fp, si);
    }
#pragma unroll
    for (int m = 0; m < NA; ++m) sh[w][m][lane] = a[m];
    __syncthreads();
    finish_rows<W>(op, sh, G, pre, blockIdx.x);
}

// resident warps per SM the tiled driver's register budget is sized for, and
// iterations of its slot loop kept in flight per warp (measured best on GB300:
// 48 warps, 2 iterations)
#ifndef TK_TILE_WARPS
#define TK_TILE_WARPS 48
#endif
#ifndef TK_TILE_UNROLL
#define TK_TILE_UNROLL 2
#endif
constexpr int kTileUnroll = TK_TILE_UNROLL;

// Ops that gather from FP32 vectors only declare kTile = n (the number of
// gathered vectors, 1 or 2), gsrc(i) (vector i) and add_t(a, k, v, s, st, si):
// the accumulation of one value times the gathered values s[0], s[st], ...
// (one tile per vector, st floats apart), with the slot's constants si.
template <class Op, class = void>
struct tile_op {
    static constexpr int value = 0;
};
template <class Op>
struct tile_op<Op, std::void_t<decltype(Op::kTile)>> {
    static constexpr int value = Op::kTile;
};

// The plain driver with the gathered vector staged in shared memory (FP32
// ops that gather from one vector).  The sources of a group lie in at most
// kTileLayers layers and in the rows y0 - H .. y1 + H of the group's first
// and last rows y0, y1; the block copies those rows of each source layer
// (whole haloed rows, coalesced) into a tile of tl floats per layer once the
// previous pass has completed, and every slot then gathers from the tile:
// tile[ttile[t] + rl], with rl the row's position within one tile layer.
// Products and their order are those of k_plain.
// One group gi of the tiled driver, shared by k_tile (one block per group,
// kPdl: the previous pass is waited for after the graph data are read) and
// the persistent batch of Chebyshev steps across requests (kCoherent: the
// gathered vector was written by other blocks of the same launch since this
// block last read it, so it is read around L1).  sh, tile, s_lay: the
// block's shared memory; a block may run several groups one after another.
template <int W, class Op, bool kPdl, bool kCoherent>
__device__ __forceinline__ void tile_group(const GridC &g, const GraphP &gp, const float *__restrict__ val,
                                           const Op &op, int gi, typename Op::A (*sh)[Op::NA][32], float *tile,
                                           int *s_lay) {
    using A = typename Op::A;
    constexpr int NA = Op::NA;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const GroupRows G = group_rows(g, gp, gi);
    // the tile's source layers are graph data: read them before waiting
    if (threadIdx.x < kTileLayers) s_lay[threadIdx.x] = __ldg(gp.tlay + G.z * kTileLayers + threadIdx.x);
    const int r0 = (gi - G.z * g.gpl) * kGroup;
    const int y0 = r0 / g.nx;
    const int y1 = min(r0 + kGroup - 1, g.nxy - 1) / g.nx;
    const int tla = (y1 - y0 + 2 * g.H + 1) * g.nxp;  // floats copied per tile layer (<= tl)
    int rl[4];
    {
        const int b = G.z * g.lp + y0 * g.nxp;
        const int pad = g.H * g.nxp + (r0 - y0 * g.nx) + g.H;  // rows past the end read the group's first row
#pragma unroll
        for (int k = 0; k < 4; ++k) rl[k] = G.row[k] >= 0 ? G.rp[k] - b : pad;
    }
    const float *v = val + G.vb + 4 * lane;
    A a[NA];
#pragma unroll
    for (int m = 0; m < NA; ++m) a[m] = A(0);
    float v0[4] = {0.f, 0.f, 0.f, 0.f}, v1[4] = {0.f, 0.f, 0.f, 0.f};
    const int tA = w, tB = w + W;
    if (tA < G.nt) ld_quad(v + (size_t)tA * kGroup, v0);
    if (tB < G.nt) ld_quad(v + (size_t)tB * kGroup, v1);
    const int ttA = tA < G.nt ? __ldg(gp.ttile + G.t0 + tA) : 0, ttB = tB < G.nt ? __ldg(gp.ttile + G.t0 + tB) : 0;
    if constexpr (kPdl) pdl_wait();
    const typename Op::Pre pre = load_pre(op, G);
    const int ts = kTileLayers * g.tl;  // floats per vector's tile
    __syncthreads();  // s_lay
#pragma unroll
    for (int iv = 0; iv < tile_op<Op>::value; ++iv) {
        const float *src = op.gsrc(iv) + (long long)y0 * g.nxp;
        for (int ls = 0; ls < kTileLayers; ++ls) {
            const int lay = s_lay[ls];
            if (lay < 0) break;  // the used tile layers come first
            const float *s = src + (long long)lay * g.lp;
            float *d = tile + iv * ts + ls * g.tl;
            for (int j = threadIdx.x; j < tla; j += 32 * W) d[j] = kCoherent ? __ldcg(s + j) : s[j];
        }
    }
    __syncthreads();
    if (tA < G.nt) {
        const auto si = op.slot(gp, G.t0 + tA);
#pragma unroll
        for (int k = 0; k < 4; ++k) op.add_t(a, k, v0[k], tile + ttA + rl[k], ts, si);
    }
    if (tB < G.nt) {
        const auto si = op.slot(gp, G.t0 + tB);
#pragma unroll
        for (int k = 0; k < 4; ++k) op.add_t(a, k, v1[k], tile + ttB + rl[k], ts, si);
    }
#pragma unroll kTileUnroll
    for (int t = w + 2 * W; t < G.nt; t += W) {
        const int tt = __ldg(gp.ttile + G.t0 + t);
        const auto si = op.slot(gp, G.t0 + t);
        float q[4];
        ld_quad(v + (size_t)t * kGroup, q);
#pragma unroll
        for (int k = 0; k < 4; ++k) op.add_t(a, k, q[k], tile + tt + rl[k], ts, si);
    }
#pragma unroll
    for (int m = 0; m < NA; ++m) sh[w][m][lane] = a[m];
    __syncthreads();
    finish_rows<W>(op, sh, G, pre, gi);
}

template <int W, class Op>
__global__ void __launch_bounds__(32 * W, TK_TILE_WARPS / W) k_tile(GridC g, GraphP gp, const float *__restrict__ val, Op op) {
    using A = typename Op::A;
    constexpr int NA = Op::NA;
    __shared__ A sh[W][NA][32];
    extern __shared__ float tile[];
    __shared__ int s_lay[kTileLayers];
    pdl_trigger();
    tile_group<W, Op, true, false>(g, gp, val, op, blockIdx.x, sh, tile, s_lay);
}

// pipelined launch: one block per run (one run per SM, at most one per group)
template <int W, class Op>
static void run_pipe(cudaStream_t st, const GridC &g, const GraphP &gp, const float *val, const Op &op, int kind) {
    const size_t smem = pipe_smem_bytes<W, typename Op::A, Op::NA>();
    static bool attr[64] = {false};  // per device: the shared-memory limit of this instantiation is raised
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(k_pipe<W, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr[dev] = true;
    }
    k_pipe<W, Op><<<gp.run_n[kind], 32 * (W + 1), smem, st>>>(g, gp, val, op, kind);
}

#ifndef TK_PDL
#define TK_PDL 1
#endif
#ifndef TK_TILE
#define TK_TILE 1
#endif
#ifndef TK_PLAIN_CARVEOUT
#define TK_PLAIN_CARVEOUT -1
#endif
template <int W, typename T, class Op>
static void run_plain(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const Op &op, int ngroups) {
#if TK_PLAIN_CARVEOUT >= 0
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(k_plain<W, T, Op>, cudaFuncAttributePreferredSharedMemoryCarveout, TK_PLAIN_CARVEOUT);
        attr[dev] = true;
    }
#endif
    // launched as a programmatic dependent of the previous work on the stream
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ngroups);
    cfg.blockDim = dim3(32 * W);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = TK_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
#if TK_TILE
    if constexpr (sizeof(T) == 4 && tile_op<Op>::value > 0) {
        const size_t tb = (size_t)tile_op<Op>::value * kTileLayers * g.tl * sizeof(float);
        if (g.tl > 0 && tb <= (size_t)kTileMaxBytes) {
            cfg.dynamicSmemBytes = tb;
            cudaLaunchKernelEx(&cfg, k_tile<W, Op>, g, gp, val, op);
            return;
        }
    }
#endif
    cudaLaunchKernelEx(&cfg, k_plain<W, T, Op>, g, gp, val, op);
}

// Dispatch on the warp count and the driver: the pipeline for FP32 scenes
// with staging on (W in {4, 8, 16}), the plain driver otherwise
// (W in {4, 6, 8, 16}).
template <typename T, class Op>
static void run_op(cudaStream_t st, const GridC &g, const GraphP &gp, const T *val, const Op &op, int kind) {
    const int ngroups = (kind == 0 ? g.nz + 1 : g.nz) * g.gpl;
    if (ngroups <= 0) return;
    if constexpr (sizeof(T) == 4) {
        if (g.stage) {
            if (g.wq == 4)
                run_pipe<4>(st, g, gp, val, op, kind);
            else if (g.wq == 8)
                run_pipe<8>(st, g, gp, val, op, kind);
            else
                run_pipe<16>(st, g, gp, val, op, kind);
            return;
        }
    }
    if (g.wq == 4)
        run_plain<4>(st, g, gp, val, op, ngroups);
    else if (g.wq == 6)
        run_plain<6>(st, g, gp, val, op, ngroups);
    else if (g.wq == 16)
        run_plain<16>(st, g, gp, val, op, ngroups);
    else
        run_plain<8>(st, g, gp, val, op, ngroups);
}

}  // namespace tk
