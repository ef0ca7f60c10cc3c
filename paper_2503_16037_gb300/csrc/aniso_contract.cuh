// The two dense contractions of the edge form (see aniso.h): the operand
// definitions (ops), the tensor-core kernel and the CUDA-core kernel.
//
// An op gives, for an atmospheric node j:
//   vraw(r, j, top), vmul(raw)   the r-th row of the per-node operand
//                 (r < R: zf X for the leave contraction, C for the sqc
//                 one), loaded raw and multiplied out when it is used
//   w(sp, j)      the species weight, so A(j, (r, sp)) = w(sp, j) v(r, j)
//   b(sp, r, n)   B((r, sp), n), an entry of the quadrature Q
//   pre(j), out(pre, j, n, value, top)   the epilogue of output n
// Leading "top" tiles of a launch (op.jtop < n_atm) cover the layers from
// which some direction has no receiver; v and out take the tile's kind.
#pragma once

#include <algorithm>
#include <type_traits>

#include <cuda.h>

#include "aniso.h"
#include "aniso_mma.cuh"
#include "asm_util.cuh"
#include "kern.h"
#include "stage.cuh"

namespace tk {

// L(u, j) = [Lsun(u, j)] + Cf(j, u) [A B](j, u) into the haloed planes, or
// (BARE, the series' folded form) G(u, j) = [A B](j, u).
// With `top` set (a second pass over the layers from which some direction
// has no receiver), A carries X without zf and only the directions without
// a receiver are written, with the routing weight 1: their light still
// crosses the source's own cell before it leaves through the top, so the
// source's self slot reads their L.
template <typename T, typename XT, typename LT, bool BARE>
struct LeaveOp {
    static constexpr bool kBatched = true;  // has out_many
    static constexpr bool bare = BARE;      // store G alone (the series' folded form), else Lsun + Cf G
    GridC g;
    int jtop;  // first node of the top layers (n_atm: no top tiles)
    const T *zf, *wsp, *CT, *on, *LsT, *Q;
    const XT *X;
    LT *Lh;
    int sun;
    int ldx, ldz;  // row strides of X and zf
    const int4 *dirs;
    // v = zf X (top tiles: X), loaded raw so that the product can wait
    struct VRaw {
        XT x;
        T z;
    };
    __device__ __forceinline__ VRaw vraw(int r, int j, bool top) const {
        return VRaw{__ldg(X + (size_t)r * ldx + j), top ? T(1) : __ldg(zf + (size_t)r * ldz + j)};
    }
    __device__ static __forceinline__ XT vmul(const VRaw &p) { return (XT)p.z * p.x; }
    __device__ __forceinline__ T w(int sp, int j) const { return __ldg(wsp + (size_t)sp * g.n_atm + j); }
    __device__ __forceinline__ T b(int sp, int r, int n) const {
        return __ldg(Q + ((size_t)sp * (g.nd + g.ngd) + r) * g.nd + n);
    }
    struct Pre {
        int x, y, z;
        long long pos;  // haloed position
        bool routed;
    };
    __device__ __forceinline__ Pre pre(int j) const {
        Pre p;
        p.z = j / g.nxy;
        const int rr = j - p.z * g.nxy;
        p.y = rr / g.nx;
        p.x = rr - p.y * g.nx;
        p.pos = halo_pos(g, p.x, p.y, p.z);
        p.routed = __ldg(on + j) > T(0);
        return p;
    }
    // main tiles write the directions with a receiver, top tiles the others
    template <typename V>
    __device__ __forceinline__ void out(const Pre &p, int j, int n, V val, bool top) const {
        const bool has = p.z + __ldg(&dirs[n].z) < g.nz;
        if (top == has) return;
        LT l = (LT)val;
        if constexpr (BARE) {
            store_halo(Lh + (size_t)n * g.npad, g, p.x, p.y, p.z, l);
        } else {
            const LT cf = (p.routed && has) ? (LT)__ldg(CT + (size_t)n * g.n_atm + j) : LT(1);
            l *= cf;
            if (sun) l += (LT)__ldg(LsT + (size_t)n * g.n_nodes + j);
            store_halo(Lh + (size_t)n * g.npad, g, p.x, p.y, p.z, l);
        }
    }
    // outputs n0 .. n0 + K - 1 (those below N): every load before the first
    // store, so that the loads of the block overlap
    template <int K, typename V>
    __device__ __forceinline__ void out_many(const Pre &p, int j, int n0, const V (&val)[K], int N,
                                             bool top) const {
        bool w[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int n = n0 + i;
            const bool in = n < N;
            const bool has = in && p.z + __ldg(&dirs[n].z) < g.nz;
            w[i] = in && top != has;
        }
        if constexpr (BARE) {
#pragma unroll
            for (int i = 0; i < K; ++i)
                if (w[i]) store_halo(Lh + (size_t)(n0 + i) * g.npad, g, p.x, p.y, p.z, (LT)val[i]);
        } else {
            LT cf[K], ls[K];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int n = n0 + i;
                const bool has = n < N && p.z + __ldg(&dirs[n].z) < g.nz;
                cf[i] = (w[i] && p.routed && has) ? (LT)__ldg(CT + (size_t)n * g.n_atm + j) : LT(1);
                ls[i] = (w[i] && sun) ? (LT)__ldg(LsT + (size_t)n * g.n_nodes + j) : LT(0);
            }
#pragma unroll
            for (int i = 0; i < K; ++i)
                if (w[i]) store_halo(Lh + (size_t)(n0 + i) * g.npad, g, p.x, p.y, p.z, cf[i] * (LT)val[i] + ls[i]);
        }
    }
};

// ops without a batched epilogue write their outputs one by one
template <class Op, int K, typename V>
__device__ __forceinline__ void out_block(const Op &op, const typename Op::Pre &p, int j, int n0, const V (&val)[K],
                                          int N, bool top) {
    if constexpr (Op::kBatched) {
        op.template out_many<K, V>(p, j, n0, val, N, top);
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i)
            if (n0 + i < N) op.out(p, j, n0 + i, val[i], top);
    }
}

// zf(w, j) = sq(j, w) / sqc(j, w) where the routing applies, else 1;
// sq from the per-layer table SQ
template <typename T>
struct SqcOp {
    static constexpr bool kBatched = false;
    GridC g;
    int jtop;  // unused (no top tiles)
    const T *CT, *wsp, *on, *SQ, *Q;
    T *zf;
    int ldz;
    struct VRaw {
        T x;
    };
    __device__ __forceinline__ VRaw vraw(int r, int j, bool) const { return VRaw{__ldg(CT + (size_t)r * g.n_atm + j)}; }
    __device__ static __forceinline__ T vmul(const VRaw &p) { return p.x; }
    __device__ __forceinline__ T w(int sp, int j) const { return __ldg(wsp + (size_t)sp * g.n_atm + j); }
    __device__ __forceinline__ T b(int sp, int r, int n) const {
        return __ldg(Q + ((size_t)sp * (g.nd + g.ngd) + n) * g.nd + r);
    }
    struct Pre {
        int z;
        bool routed;
        T ws[MAX_SPECIES];
    };
    __device__ __forceinline__ Pre pre(int j) const {
        Pre p;
        p.z = j / g.nxy;
        p.routed = __ldg(on + j) > T(0);
#pragma unroll
        for (int sp = 0; sp < MAX_SPECIES; ++sp) p.ws[sp] = sp < g.S ? w(sp, j) : T(0);
        return p;
    }
    template <typename V>
    __device__ __forceinline__ void out(const Pre &p, int j, int n, V val, bool) const {
        T z = T(1);
        if (p.routed && val > V(0)) {
            const int nin = g.nd + g.ngd;
            T sq = T(0);
#pragma unroll
            for (int sp = 0; sp < MAX_SPECIES; ++sp)
                if (sp < g.S) sq += p.ws[sp] * __ldg(SQ + ((size_t)p.z * g.S + sp) * nin + n);
            z = sq / (T)val;
        }
        zf[(size_t)n * ldz + j] = z;
    }
};

// ---- tensor cores ----
// Shared memory of one launch: a ring of NS stages, each A (high, low) and
// B (high, low) of one K chunk, and a ring of NR stages of the raw X and zf
// boxes of a chunk (tensor-map copies); padded so that the blocks an SM can
// hold never ask for more than the 512 columns of tensor memory (two
// accumulators of np columns each per block).
template <int S, int NP>
struct MmaShape {
    static constexpr int KC = kAniRows * S;
    static constexpr int NR = 4;  // raw X / zf stages (tensor-map copies run this far ahead)
    static constexpr unsigned A_BYTES = 128u * KC * 4;
    static constexpr unsigned B_BYTES = (unsigned)NP * KC * 4;
    static constexpr unsigned STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr unsigned RAW_HALF = kAniRows * 128u * 4;  // one box: kAniRows rows x 128 nodes
    static constexpr unsigned RAW = 2 * RAW_HALF;              // X, then zf
    // A/B stages: as many as fit beside the raw ring in about 200 KB (up to
    // 4), so that the MMAs' completion is rarely waited for
    static constexpr int NS_FIT = (int)((200u * 1024u - NR * RAW) / STAGE);
    static constexpr int NS = NS_FIT < 2 ? 2 : (NS_FIT > 4 ? 4 : NS_FIT);
    static constexpr unsigned RAW_OFF = NS * STAGE;
    static constexpr unsigned ACOLS = NP <= 32 ? 32 : NP <= 64 ? 64 : NP <= 128 ? 128 : 256;
    static constexpr unsigned TCOLS = 2 * ACOLS;
    static constexpr unsigned MAXC = 512 / TCOLS;
    static constexpr unsigned PAD = (233472u / (MAXC + 1) + 1024u) / 1024u * 1024u;
    static constexpr unsigned NEED = RAW_OFF + NR * RAW;
    static constexpr unsigned SMEM = NEED > PAD ? NEED : PAD;
    static_assert(RAW_OFF % 1024 == 0, "raw ring alignment");
};

// Bounded wait for the phase of the given parity: a few non-blocking tests
// (a phase that is about to complete), then mbarrier.try_wait, which parks
// the thread until the phase completes (or for a few microseconds), so that
// waiting warps take neither issue slots nor shared-memory bandwidth from
// the working ones; about a second in all.  False after giving up
// (STATUS_TIMEOUT and the block's abort flag set), or at once once the block
// has aborted when honour_abort is set.
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
static __device__ __noinline__ bool spin_wait(unsigned bar, unsigned parity, int *abort_flag, int *status,
                                              bool honour_abort) {
    for (int i = 0; i < 16; ++i)
        if (mbar_test(bar, parity)) return true;
    return pipe_wait(bar, parity, abort_flag, status, honour_abort);
}
// announce `bytes` of transfer on the barrier (without arriving)
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// one arrival that also announces `bytes` of transfer
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// one box of a 2-D tensor map (coordinates x inner, y outer; x * 4 bytes a
// multiple of 16) into shared memory, counted in bytes on the barrier
__device__ __forceinline__ void tensor_copy_2d(unsigned bar, unsigned dst, const CUtensorMap *map, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bulk_copy(unsigned bar, unsigned dst, const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Persistent, warp-specialised tensor-core contraction of the leave op (v =
// zf X; top tiles: X).  Tiles of 128 nodes (the first ntop are the top
// layers' tiles, from op.jtop, a multiple of 128) are dealt to the blocks
// round robin.  Fourteen warps (P = kMmaProducerWarps = 8):
//   P+5  its lane 0 copies each chunk's X and zf boxes (kAniRows rows x 128
//        nodes, tensor maps mx, mz; zero beyond the arrays) into the raw
//        ring, up to NR chunks ahead
//   0..P-1  producers: threads m and m + 128 own row m of A, each half of
//        the chunk's rows of v; per K chunk a thread reads its raw values,
//        releases the raw stage, waits for a free A/B stage, stores w v split
//        in TF32 high and low parts in the core-matrix layout and arrives on
//        the stage's full barrier (thread 0 first starts the copy of the
//        chunk's packed B into the stage, counted in bytes on the same
//        barrier)
//   P..P+3  epilogue: drain one of the two tensor-memory accumulators (warp
//        w reads lanes 32 (w % 4) ..) and write the outputs, then release it
//   P+4  its lane 0 issues the 3 kc / 8 MMAs of each chunk once its stage is
//        full, commits them to the stage's empty barrier, and after a tile's
//        last chunk to the accumulator's full barrier
// Waits are bounded; after a timeout every wait that may return at once
// does, no MMA is issued, every barrier still gets its arrivals, and the
// block waits for its copies, frees its tensor memory and returns with
// STATUS_TIMEOUT set.
constexpr int kMmaProducerWarps = 8;  // two threads per row of A, each half of a chunk's rows of v
constexpr int kMmaThreads = 32 * (kMmaProducerWarps + 6);
template <int S, int NP, class Op>
__global__ void __launch_bounds__(kMmaThreads, 1) k_ani_mma(Op op, int R, int N, int ntop, int ntiles,
                                                            const float *__restrict__ Btab,
                                                            const __grid_constant__ CUtensorMap mx,
                                                            const __grid_constant__ CUtensorMap mz, const int *ctl,
                                                            int *status) {
    using Sh = MmaShape<S, NP>;
    constexpr int KC = Sh::KC, NS = Sh::NS, NR = Sh::NR;
    constexpr uint32_t kIdesc = umma_idesc_tf32(128, NP);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long full[NS], empty[NS], rfull[NR], rempty[NR], accf[2], acce[2];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    if (ctl && *(volatile const int *)ctl) return;  // the series has converged
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = ani_chunks(R);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_addr(&full[s]), 32 * kMmaProducerWarps);
            mbar_init(smem_addr(&empty[s]), 1);
        }
        for (int s = 0; s < NR; ++s) {
            mbar_init(smem_addr(&rfull[s]), 1);
            mbar_init(smem_addr(&rempty[s]), 32 * kMmaProducerWarps);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_addr(&accf[a]), 1);
            mbar_init(smem_addr(&acce[a]), 128);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_addr(&tmem_slot), Sh::TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;
    const unsigned sbase = smem_addr(smem);
    const float *raw = reinterpret_cast<const float *>(smem + Sh::RAW_OFF);
    auto tile_j0 = [&](int t, bool &top) {
        top = t < ntop;
        return top ? op.jtop + t * kAniTileM : (t - ntop) * kAniTileM;
    };
    if (warp < kMmaProducerWarps) {
        // ---- producers: thread (m, h) = (tid % 128, tid / 128) stages the
        // K values of row m that come from rows h RH .. h RH + RH - 1 of v ----
        constexpr int RH = kAniRows / 2, KH = RH * S;
        const int m = tid & 127, h = tid >> 7;
        int q = 0;  // chunks staged by this block so far
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            bool top;
            const int j = tile_j0(t, top) + m;
            const bool valid = j < op.g.n_atm;
            float ws[S];
#pragma unroll
            for (int sp = 0; sp < S; ++sp) ws[sp] = valid ? (float)op.w(sp, j) : 0.f;
            for (int c = 0; c < nch; ++c, ++q) {
                const int rs = q % NR, slot = q % NS;
                spin_wait(smem_addr(&rfull[rs]), (unsigned)((q / NR) & 1), &abort_flag, status, true);
                const float *rx = raw + rs * (Sh::RAW / 4) + h * RH * 128 + m, *rz = rx + Sh::RAW_HALF / 4;
                float vc[RH];
#pragma unroll
                for (int i = 0; i < RH; ++i) vc[i] = top ? rx[i * 128] : rz[i * 128] * rx[i * 128];
                mbar_arrive(smem_addr(&rempty[rs]));
                const unsigned st = sbase + slot * Sh::STAGE;
                spin_wait(smem_addr(&empty[slot]), (unsigned)(((q / NS) & 1) ^ 1), &abort_flag, status, true);
                if (tid == 0) {
                    mbar_expect_tx(smem_addr(&full[slot]), 2 * Sh::B_BYTES);
                    bulk_copy(smem_addr(&full[slot]), st + 2 * Sh::A_BYTES, Btab + (size_t)c * 2 * NP * KC,
                              2 * Sh::B_BYTES);
                }
#pragma unroll
                for (int k4 = 0; k4 < KH / 4; ++k4) {
                    float hi[4], lo[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int k = 4 * k4 + e;  // K index h KH + k of the chunk
                        const float a = ws[k % S] * vc[k / S];
                        hi[e] = tf32_rna(a);
                        lo[e] = tf32_rna(a - hi[e]);
                    }
                    const unsigned off = op_offset<KC>(m, h * KH + 4 * k4);
                    st_shared_v4(st + off, hi[0], hi[1], hi[2], hi[3]);
                    st_shared_v4(st + Sh::A_BYTES + off, lo[0], lo[1], lo[2], lo[3]);
                }
                fence_async_smem();
                mbar_arrive(smem_addr(&full[slot]));
            }
        }
    } else if (warp < kMmaProducerWarps + 4) {
        // ---- epilogue ----
        const int quarter = warp & 3;
        int lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            bool top;
            const int j = tile_j0(t, top) + 32 * quarter + lane;
            const bool valid = j < op.g.n_atm;
            const int acc = lt & 1;
            spin_wait(smem_addr(&accf[acc]), (unsigned)((lt >> 1) & 1), &abort_flag, status, true);
            tc_fence_after();
            const typename Op::Pre pr = op.pre(valid ? j : 0);
            const unsigned ta = tmem + acc * Sh::ACOLS + ((unsigned)(32 * quarter) << 16);
#pragma unroll 1
            for (int ck = 0; ck < NP / 16; ++ck) {
                float o[16];
                __syncwarp();  // tcgen05.ld is warp-wide
                tmem_ld16(ta + (unsigned)(16 * ck), o);
                if (valid) out_block(op, pr, j, 16 * ck, o, N, top);
            }
            tc_fence_before();
            mbar_arrive(smem_addr(&acce[acc]));
        }
    } else if (warp == kMmaProducerWarps + 4) {
        // ---- MMA issue (the whole warp walks the loop, lane 0 acts) ----
        int q = 0, lt = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
            const int acc = lt & 1;
            // the epilogue has drained this accumulator (tile lt - 2)
            if (lane == 0)
                spin_wait(smem_addr(&acce[acc]), (unsigned)(((lt >> 1) & 1) ^ 1), &abort_flag, status, true);
            __syncwarp();
            tc_fence_after();
            const unsigned d = tmem + acc * Sh::ACOLS;
            for (int c = 0; c < nch; ++c, ++q) {
                const int slot = q % NS;
                const unsigned st = sbase + slot * Sh::STAGE;
                if (lane == 0) spin_wait(smem_addr(&full[slot]), (unsigned)((q / NS) & 1), &abort_flag, status, false);
                __syncwarp();
                tc_fence_after();
                if (lane == 0 && !*(volatile int *)&abort_flag) {
                    // a K step of 8 is 32 bytes along the row (swizzled) or two core matrices
                    constexpr unsigned kStep = sw_mode(KC) ? 32u : 256u;
#pragma unroll
                    for (int ks = 0; ks < KC / 8; ++ks) {
                        const unsigned ah = st + kStep * ks, al = ah + Sh::A_BYTES;
                        const unsigned bh = st + 2 * Sh::A_BYTES + kStep * ks, bl = bh + Sh::B_BYTES;
                        const uint64_t dah = op_desc<KC>(ah), dal = op_desc<KC>(al);
                        const uint64_t dbh = op_desc<KC>(bh), dbl = op_desc<KC>(bl);
                        umma_tf32(d, dah, dbh, kIdesc, (c | ks) != 0);
                        umma_tf32(d, dah, dbl, kIdesc, 1);
                        umma_tf32(d, dal, dbh, kIdesc, 1);
                    }
                }
                if (lane == 0) umma_commit(smem_addr(&empty[slot]));
                __syncwarp();
            }
            if (lane == 0) umma_commit(smem_addr(&accf[acc]));
            __syncwarp();
        }
    } else {
        // ---- raw copies (the whole warp walks the loop, lane 0 acts) ----
        int q = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            bool top;
            const int j0 = tile_j0(t, top);
            for (int c = 0; c < nch; ++c, ++q) {
                const int rs = q % NR;
                if (lane == 0) {
                    spin_wait(smem_addr(&rempty[rs]), (unsigned)(((q / NR) & 1) ^ 1), &abort_flag, status, true);
                    const unsigned dst = sbase + Sh::RAW_OFF + rs * Sh::RAW;
                    mbar_arrive_expect_tx(smem_addr(&rfull[rs]), top ? Sh::RAW_HALF : Sh::RAW);
                    tensor_copy_2d(smem_addr(&rfull[rs]), dst, &mx, j0, c * kAniRows);
                    if (!top) tensor_copy_2d(smem_addr(&rfull[rs]), dst + Sh::RAW_HALF, &mz, j0, c * kAniRows);
                }
                __syncwarp();
            }
        }
        // every copy of this warp has landed before the block ends
        if (lane == 0)
            for (int i = q - NR > 0 ? q - NR : 0; i < q; ++i)
                spin_wait(smem_addr(&rfull[i % NR]), (unsigned)((i / NR) & 1), &abort_flag, status, false);
        __syncwarp();
    }
    // every MMA completed before the epilogue's last wait; every copy was
    // waited for by the MMA and the copy warps
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, Sh::TCOLS);
}

// packed B of the tensor-core kernel: per chunk, high then low parts, each
// np x kc in the operand layout of op_offset (entries past R or N are 0)
template <class Op, int KC>
__global__ void k_ani_pack(Op op, int R, int N, int np, float *Btab) {
    constexpr int S = KC / kAniRows, kc = KC;
    const long long per = (long long)np * kc;
    const long long total = (long long)ani_chunks(R) * per;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(idx / per);
        const int rem = (int)(idx - (long long)c * per);
        const int n = rem / kc, k = rem - n * kc;
        const int r = c * kAniRows + k / S, sp = k % S;
        const float b = (r < R && n < N) ? (float)op.b(sp, r, n) : 0.f;
        const float h = tf32_rna(b), l = tf32_rna(b - h);
        float *base = Btab + (size_t)c * 2 * per;
        const unsigned o = op_offset<KC>(n, k) >> 2;
        base[o] = h;
        base[per + o] = l;
    }
}

// ---- CUDA cores ----
// double-single accumulation: (sh, sl) += (ah + al) b with the product ah b
// exact (FMA) and the sum compensated (two-sum)
__device__ __forceinline__ void ds_fma(float &sh, float &sl, float ah, float al, float b) {
    const float p = __fmul_rn(ah, b);
    const float e = __fmaf_rn(ah, b, -p);
    const float t = __fadd_rn(sh, p);
    const float bb = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    sh = t;
    sl = __fmaf_rn(al, b, __fadd_rn(sl, __fadd_rn(err, e)));
}

// Tile of 64 nodes x 128 outputs (blockIdx.y: the column block), 256
// threads: thread (tx, ty) = (tid % 16, tid / 16) accumulates nodes
// 4 tx .. 4 tx + 3 times outputs 8 ty .. 8 ty + 7, in T.  Per chunk the
// block loads every operand value first, then stages A (kc x 64) and B
// (kc x 128) in shared memory.
constexpr int kSimtM = 64, kSimtN = 128;
template <typename T, class Op>
__global__ void __launch_bounds__(256) k_ani_simt(Op op, int S, int R, int N, int ntop, const int *ctl) {
    extern __shared__ __align__(16) unsigned char smem_s[];
    if (ctl && *(volatile const int *)ctl) return;
    const int kc = kAniRows * S;
    T *As = (T *)smem_s;                                     // [kc][64]
    T *Bs = (T *)(smem_s + (size_t)kc * kSimtM * sizeof(T));  // [kc][128]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const bool top = (int)blockIdx.x < ntop;
    const int j0 = top ? op.jtop + (int)blockIdx.x * kSimtM : ((int)blockIdx.x - ntop) * kSimtM;
    const int n0 = blockIdx.y * kSimtN;
    T acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = T(0);
    const int nch = ani_chunks(R);
    for (int c = 0; c < nch; ++c) {
        constexpr int kLa = 2 * MAX_SPECIES, kLb = 4 * MAX_SPECIES;  // kc 64 / 256 and kc 128 / 256 at most
        typename Op::VRaw ra[kLa];
        T wa[kLa], rb[kLb];
#pragma unroll
        for (int it = 0; it < kLa; ++it) {
            const int idx = tid + 256 * it;
            const int k = idx >> 6, jj = j0 + (idx & 63);
            const int r = c * kAniRows + k / S, sp = k % S;
            const bool ok = it < 2 * S && jj < op.g.n_atm && r < R;
            ra[it] = ok ? op.vraw(r, jj, top) : typename Op::VRaw{};
            wa[it] = ok ? op.w(sp, jj) : T(0);
        }
#pragma unroll
        for (int it = 0; it < kLb; ++it) {
            const int idx = tid + 256 * it;
            const int k = idx >> 7, n = n0 + (idx & 127);
            const int r = c * kAniRows + k / S, sp = k % S;
            rb[it] = (it < 4 * S && r < R && n < N) ? op.b(sp, r, n) : T(0);
        }
        __syncthreads();  // the previous chunk is read
#pragma unroll
        for (int it = 0; it < kLa; ++it)
            if (it < 2 * S) As[tid + 256 * it] = wa[it] * (T)Op::vmul(ra[it]);
#pragma unroll
        for (int it = 0; it < kLb; ++it)
            if (it < 4 * S) Bs[tid + 256 * it] = rb[it];
        __syncthreads();
        if (n0 + 8 * ty < N)  // column groups entirely past N have nothing to add
#pragma unroll 2
            for (int k = 0; k < kc; ++k) {
                T a[4], b[8];
#pragma unroll
                for (int q = 0; q < 4; ++q) a[q] = As[k * kSimtM + 4 * tx + q];
#pragma unroll
                for (int q = 0; q < 8; ++q) b[q] = Bs[k * kSimtN + 8 * ty + q];
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[p][q] += a[p] * b[q];
            }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int j = j0 + 4 * tx + p;
        if (j >= op.g.n_atm) continue;
        const typename Op::Pre pr = op.pre(j);
        out_block(op, pr, j, n0 + 8 * ty, acc[p], N, top);
    }
}

template <typename T>
inline size_t ani_simt_smem(int S) {
    const int kc = kAniRows * S;
    return (size_t)kc * kSimtM * sizeof(T) + (size_t)kc * kSimtN * sizeof(T);
}

// the main tiles, preceded by the top layers' tiles when op.jtop < n_atm
template <typename T, class Op>
inline void ani_simt_launch(cudaStream_t st, const Op &op, int S, int R, int N, const int *ctl) {
    const size_t sm = ani_simt_smem<T>(S);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_ani_simt<T, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int ntop = op.jtop < op.g.n_atm ? (op.g.n_atm - op.jtop + kSimtM - 1) / kSimtM : 0;
    const dim3 grid(ntop + (op.g.n_atm + kSimtM - 1) / kSimtM, (N + kSimtN - 1) / kSimtN);
    k_ani_simt<T, Op><<<grid, 256, sm, st>>>(op, S, R, N, ntop, ctl);
}

template <int S, int NP, class Op>
inline void ani_mma_launch(cudaStream_t st, const Op &op, int R, int N, const float *Btab, const CUtensorMap &mx,
                           const CUtensorMap &mz, const int *ctl, int *status) {
    using Sh = MmaShape<S, NP>;
    static int grid_max = 0;  // blocks the GPU holds at once (per instantiation)
    if (grid_max == 0) {
        cudaFuncSetAttribute(k_ani_mma<S, NP, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
        cudaFuncSetAttribute(k_ani_mma<S, NP, Op>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        int dev = 0, nsm = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ani_mma<S, NP, Op>, kMmaThreads, Sh::SMEM);
        grid_max = std::max(1, nsm * std::max(1, per));
    }
    const int ntop = op.jtop < op.g.n_atm ? (op.g.n_atm - op.jtop + kAniTileM - 1) / kAniTileM : 0;
    const int ntiles = ntop + (op.g.n_atm + kAniTileM - 1) / kAniTileM;
    k_ani_mma<S, NP, Op><<<std::min(ntiles, grid_max), kMmaThreads, Sh::SMEM, st>>>(op, R, N, ntop, ntiles, Btab, mx,
                                                                                   mz, ctl, status);
}

}  // namespace tk
