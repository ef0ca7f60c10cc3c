// The two dense contractions of the edge form (see aniso.h): the operand
// definitions (ops), the tensor-core kernel and the CUDA-core kernel.
//
// An op gives, for an atmospheric node j:
//   v(r, j)       the r-th row of the per-node operand (r < R: zf X for the
//                 leave contraction, C for the sqc one)
//   w(sp, j)      the species weight, so A(j, (r, sp)) = w(sp, j) v(r, j)
//   b(sp, r, n)   B((r, sp), n), an entry of the quadrature Q
//   pre(j), out(pre, j, n, value)   the epilogue of output n
#pragma once

#include <type_traits>

#include "aniso.h"
#include "aniso_mma.cuh"
#include "asm_util.cuh"
#include "kern.h"
#include "stage.cuh"

namespace tk {

// L(u, j) = [Lsun(u, j)] + Cf(j, u) [A B](j, u) into the haloed planes.
// With `top` set (a second pass over the layers from which some direction
// has no receiver), A carries X without zf and only the directions without
// a receiver are written, with the routing weight 1: their light still
// crosses the source's own cell before it leaves through the top, so the
// source's self slot reads their L.
template <typename T, typename XT, typename LT>
struct LeaveOp {
    GridC g;
    int jbeg;  // first node of the pass
    const T *zf, *wsp, *CT, *on, *LsT, *Q;
    const XT *X;
    LT *Lh;
    int sun, top;
    const int4 *dirs;
    __device__ __forceinline__ XT v(int r, int j) const {
        const XT x = __ldg(X + (size_t)r * g.n_nodes + j);
        return top ? x : (XT)__ldg(zf + (size_t)r * g.n_atm + j) * x;
    }
    __device__ __forceinline__ T w(int sp, int j) const { return __ldg(wsp + (size_t)sp * g.n_atm + j); }
    __device__ __forceinline__ T b(int sp, int r, int n) const {
        return __ldg(Q + ((size_t)sp * (g.nd + g.ngd) + r) * g.nd + n);
    }
    struct Pre {
        int x, y, z;
        bool routed;
    };
    __device__ __forceinline__ Pre pre(int j) const {
        Pre p;
        p.z = j / g.nxy;
        const int rr = j - p.z * g.nxy;
        p.y = rr / g.nx;
        p.x = rr - p.y * g.nx;
        p.routed = __ldg(on + j) > T(0);
        return p;
    }
    template <typename V>
    __device__ __forceinline__ void out(const Pre &p, int j, int n, V val) const {
        const bool has = p.z + __ldg(&dirs[n].z) < g.nz;
        if (top && has) return;
        const LT cf = (p.routed && has) ? (LT)__ldg(CT + (size_t)n * g.n_atm + j) : LT(1);
        LT l = cf * (LT)val;
        if (sun) l += (LT)__ldg(LsT + (size_t)n * g.n_nodes + j);
        store_halo(Lh + (size_t)n * g.npad, g, p.x, p.y, p.z, l);
    }
};

// zf(w, j) = sq(j, w) / sqc(j, w) where the routing applies, else 1;
// sq from the per-layer table SQ
template <typename T>
struct SqcOp {
    GridC g;
    int jbeg;
    const T *CT, *wsp, *on, *SQ, *Q;
    T *zf;
    __device__ __forceinline__ T v(int r, int j) const { return __ldg(CT + (size_t)r * g.n_atm + j); }
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
    __device__ __forceinline__ void out(const Pre &p, int j, int n, V val) const {
        T z = T(1);
        if (p.routed && val > V(0)) {
            const int nin = g.nd + g.ngd;
            T sq = T(0);
#pragma unroll
            for (int sp = 0; sp < MAX_SPECIES; ++sp)
                if (sp < g.S) sq += p.ws[sp] * __ldg(SQ + ((size_t)p.z * g.S + sp) * nin + n);
            z = sq / (T)val;
        }
        zf[(size_t)n * g.n_atm + j] = z;
    }
};

// ---- tensor cores ----
// Shared memory of one launch: two stages, each A high, A low, B high, B
// low; padded so that the blocks an SM can hold never ask for more than the
// 512 columns of tensor memory.
template <int S, int NP>
struct MmaShape {
    static constexpr int KC = kAniRows * S;
    static constexpr unsigned A_BYTES = 128u * KC * 4;
    static constexpr unsigned B_BYTES = (unsigned)NP * KC * 4;
    static constexpr unsigned STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr unsigned TCOLS = NP <= 32 ? 32 : NP <= 64 ? 64 : NP <= 128 ? 128 : 256;
    static constexpr unsigned MAXC = 512 / TCOLS;
    static constexpr unsigned PAD = (233472u / (MAXC + 1) + 1024u) / 1024u * 1024u;
    static constexpr unsigned SMEM = 2 * STAGE > PAD ? 2 * STAGE : PAD;
};

// One block per 128-node tile.  Every thread owns one row (node) of A: it
// loads its kAniRows values of v per chunk (the next chunk's while the
// current one's MMAs run), splits w v into TF32 high and low parts and
// stores them in the core-matrix layout; one thread copies the chunk's
// packed B (cp.async.bulk), issues the 3 kc / 8 MMAs and commits them to the
// stage's mbarrier.  Waits are bounded (pipe_wait); after a timeout the
// block issues no more MMAs, still commits, waits for its copies and MMAs,
// frees its tensor memory and returns with STATUS_TIMEOUT set.
template <int S, int NP, class Op>
__global__ void __launch_bounds__(128) k_ani_mma(Op op, int R, int N, const float *__restrict__ Btab,
                                                 const int *ctl, int *status) {
    using Sh = MmaShape<S, NP>;
    constexpr int KC = Sh::KC;
    constexpr uint32_t kIdesc = umma_idesc_tf32(128, NP);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar_b[2], bar_m[2];
    __shared__ unsigned tmem_slot;
    __shared__ int abort_flag;
    if (ctl && *(volatile const int *)ctl) return;  // the series has converged
    const int tid = threadIdx.x, wq = tid >> 5;
    const int j = op.jbeg + blockIdx.x * kAniTileM + tid;
    const bool valid = j < op.g.n_atm;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_addr(&bar_b[s]), 1);
            mbar_init(smem_addr(&bar_m[s]), 1);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (wq == 0) tmem_alloc(smem_addr(&tmem_slot), Sh::TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;
    const unsigned sbase = smem_addr(smem);
    float ws[S];
#pragma unroll
    for (int sp = 0; sp < S; ++sp) ws[sp] = valid ? (float)op.w(sp, j) : 0.f;
    const int nch = ani_chunks(R);
    float v[kAniRows];
    auto load = [&](int c) {
#pragma unroll
        for (int i = 0; i < kAniRows; ++i) {
            const int r = c * kAniRows + i;
            v[i] = (valid && r < R) ? (float)op.v(r, j) : 0.f;
        }
    };
    load(0);
    unsigned pm = 0, pb = 0;  // parity of the next phase to wait for, per stage (bit s)
    for (int c = 0; c < nch; ++c) {
        const int s = c & 1;
        const unsigned st = sbase + s * Sh::STAGE;
        if (c >= 2) {  // the stage's previous MMAs have read it
            pipe_wait(smem_addr(&bar_m[s]), (pm >> s) & 1u, &abort_flag, status, true);
            pm ^= 1u << s;
        }
        if (tid == 0)
            bulk_load(smem_addr(&bar_b[s]), smem + s * Sh::STAGE + 2 * Sh::A_BYTES,
                      Btab + (size_t)c * 2 * NP * KC, 2 * Sh::B_BYTES);
#pragma unroll
        for (int q = 0; q < KC / 4; ++q) {
            float h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * q + e;
                const float a = ws[k % S] * v[k / S];
                h[e] = tf32_rna(a);
                l[e] = tf32_rna(a - h[e]);
            }
            const unsigned off = cm_offset(tid, 4 * q, KC);
            st_shared_v4(st + off, h[0], h[1], h[2], h[3]);
            st_shared_v4(st + Sh::A_BYTES + off, l[0], l[1], l[2], l[3]);
        }
        fence_async_smem();
        if (c + 1 < nch) load(c + 1);
        __syncthreads();
        if (tid == 0) {
            pipe_wait(smem_addr(&bar_b[s]), (pb >> s) & 1u, &abort_flag, status, false);
            pb ^= 1u << s;
            tc_fence_after();
            if (!*(volatile int *)&abort_flag) {
                constexpr unsigned kSbo = 32u * KC;
#pragma unroll
                for (int ks = 0; ks < KC / 8; ++ks) {
                    const unsigned ah = st + 256u * ks, al = ah + Sh::A_BYTES;
                    const unsigned bh = st + 2 * Sh::A_BYTES + 256u * ks, bl = bh + Sh::B_BYTES;
                    umma_tf32(tmem, umma_desc(ah, 128, kSbo), umma_desc(bh, 128, kSbo), kIdesc, (c | ks) != 0);
                    umma_tf32(tmem, umma_desc(ah, 128, kSbo), umma_desc(bl, 128, kSbo), kIdesc, 1);
                    umma_tf32(tmem, umma_desc(al, 128, kSbo), umma_desc(bh, 128, kSbo), kIdesc, 1);
                }
            }
            umma_commit(smem_addr(&bar_m[s]));
        }
    }
    {  // the last commit covers every MMA of the block
        const int s = (nch - 1) & 1;
        pipe_wait(smem_addr(&bar_m[s]), (pm >> s) & 1u, &abort_flag, status, false);
    }
    tc_fence_after();
    const typename Op::Pre pr = op.pre(valid ? j : op.jbeg);
#pragma unroll 1
    for (int col = 0; col < NP; col += 16) {
        float o[16];
        tmem_ld16(tmem + ((unsigned)(wq * 32) << 16) + (unsigned)col, o);
        if (valid) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (col + i < N) op.out(pr, j, col + i, o[i]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (wq == 0) tmem_dealloc(tmem, Sh::TCOLS);
}

// packed B of the tensor-core kernel: per chunk, high then low parts, each
// np x kc in the core-matrix layout (entries past R or N are 0)
template <class Op>
__global__ void k_ani_pack(Op op, int S, int R, int N, int np, float *Btab) {
    const int kc = kAniRows * S;
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
        const unsigned o = cm_offset(n, k, kc) >> 2;
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

// Tile of 32 nodes x all N outputs, 256 threads: thread (m, cg) accumulates
// node m's outputs n = cg + 8 q.  Per chunk the block stages A (32 x kc) and
// B (kc x N) in shared memory.  MODE 0: arithmetic in T; MODE 1 (T = float):
// v in FP64, A split in FP32 pairs, products accumulated in double-single.
constexpr int kSimtQ = 32;  // outputs per thread: N <= 8 kSimtQ
template <typename T, int MODE, class Op>
__global__ void __launch_bounds__(256) k_ani_simt(Op op, int S, int R, int N, const int *ctl) {
    using AT = typename std::conditional<MODE == 1, float2, T>::type;
    extern __shared__ __align__(16) unsigned char smem_s[];
    if (ctl && *(volatile const int *)ctl) return;
    const int kc = kAniRows * S;
    AT *As = (AT *)smem_s;                 // [kc][32]
    T *Bs = (T *)(smem_s + (size_t)kc * 32 * sizeof(AT));  // [kc][N]
    const int tid = threadIdx.x, m = tid & 31, cg = tid >> 5;
    const int j0 = op.jbeg + blockIdx.x * 32;
    T acc[kSimtQ], acl[kSimtQ];
#pragma unroll
    for (int q = 0; q < kSimtQ; ++q) acc[q] = acl[q] = T(0);
    const int nch = ani_chunks(R);
    for (int c = 0; c < nch; ++c) {
        __syncthreads();
        for (int idx = tid; idx < kc * 32; idx += 256) {
            const int k = idx >> 5, mm = idx & 31, jj = j0 + mm;
            const int r = c * kAniRows + k / S, sp = k % S;
            const bool ok = jj < op.g.n_atm && r < R;
            if constexpr (MODE == 1) {
                const double a = ok ? (double)op.w(sp, jj) * op.v(r, jj) : 0.0;
                const float ah = (float)a;
                As[idx] = make_float2(ah, (float)(a - (double)ah));
            } else {
                As[idx] = ok ? op.w(sp, jj) * (T)op.v(r, jj) : T(0);
            }
        }
        for (int idx = tid; idx < kc * N; idx += 256) {
            const int k = idx / N, n = idx - k * N;
            const int r = c * kAniRows + k / S, sp = k % S;
            Bs[idx] = r < R ? op.b(sp, r, n) : T(0);
        }
        __syncthreads();
        for (int k = 0; k < kc; ++k) {
            const AT a = As[k * 32 + m];
            const T *br = Bs + (size_t)k * N;
#pragma unroll
            for (int q = 0; q < kSimtQ; ++q) {
                const int n = cg + 8 * q;
                if (n < N) {
                    if constexpr (MODE == 1) ds_fma(acc[q], acl[q], a.x, a.y, br[n]);
                    else acc[q] += a * br[n];
                }
            }
        }
    }
    const int j = j0 + m;
    if (j >= op.g.n_atm) return;
    const typename Op::Pre pr = op.pre(j);
#pragma unroll
    for (int q = 0; q < kSimtQ; ++q) {
        const int n = cg + 8 * q;
        if (n < N) {
            if constexpr (MODE == 1) op.out(pr, j, n, (double)acc[q] + (double)acl[q]);
            else op.out(pr, j, n, acc[q]);
        }
    }
}

template <typename T, int MODE>
inline size_t ani_simt_smem(int S, int N) {
    using AT = typename std::conditional<MODE == 1, float2, T>::type;
    const int kc = kAniRows * S;
    return (size_t)kc * 32 * sizeof(AT) + (size_t)kc * N * sizeof(T);
}

template <typename T, int MODE, class Op>
inline void ani_simt_launch(cudaStream_t st, const Op &op, int S, int R, int N, const int *ctl) {
    const size_t sm = ani_simt_smem<T, MODE>(S, N);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_ani_simt<T, MODE, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (op.jbeg >= op.g.n_atm) return;
    k_ani_simt<T, MODE, Op><<<(op.g.n_atm - op.jbeg + 31) / 32, 256, sm, st>>>(op, S, R, N, ctl);
}

template <int S, int NP, class Op>
inline void ani_mma_launch(cudaStream_t st, const Op &op, int R, int N, const float *Btab, const int *ctl,
                           int *status) {
    using Sh = MmaShape<S, NP>;
    cudaFuncSetAttribute(k_ani_mma<S, NP, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
    if (op.jbeg >= op.g.n_atm) return;
    k_ani_mma<S, NP, Op><<<(op.g.n_atm - op.jbeg + kAniTileM - 1) / kAniTileM, 128, Sh::SMEM, st>>>(
        op, R, N, Btab, ctl, status);
}

}  // namespace tk
