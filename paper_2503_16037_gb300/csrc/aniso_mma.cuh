// Dense contractions of the edge form on the tensor cores (tcgen05, sm_103a).
//
// out(j, n) = sum_k A(j, k) B(k, n) over a tile of kAniTileM = 128 nodes j
// (the MMA's M) and all np outputs n (its N), K in chunks of kc = kAniRows S
// values.  FP32 operands are split as a = hi + lo with hi, lo rounded to TF32
// and the three products hi*hi + hi*lo + lo*hi accumulate in FP32 in tensor
// memory (the dropped lo*lo term is 2^-22 of the product).
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// 8 x 16-byte core matrices (8 rows, 4 TF32 values of K each), the core
// matrices of one row group adjacent along K (leading offset 128 bytes), row
// groups kc / 4 core matrices apart (stride offset 32 kc bytes).  One MMA
// takes K = 8, two core matrices along K.  The accumulator lives in tensor
// memory: row m of the tile in lane m, output n in column n.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace tk {

__device__ __forceinline__ float tf32_rna(float a) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
    return __uint_as_float(r);
}

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), the descriptor version bit (46) of tcgen05, no swizzle
__device__ __forceinline__ uint64_t umma_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1),
// A and B TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(unsigned tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on the mbarrier once every tcgen05 operation this thread issued so
// far has completed
__device__ __forceinline__ void umma_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(unsigned dst_smem, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(unsigned tmem, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// generic-proxy shared-memory writes become visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 16 columns of 32 bits: thread t of the warp gets lane
// (base lane + t), columns col .. col + 15
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void st_shared_v4(unsigned addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// byte offset of element (row, k) in a K-major no-swizzle operand of kc
// values per row
__host__ __device__ __forceinline__ unsigned cm_offset(int row, int k, int kc) {
    return (unsigned)((((row >> 3) * (kc >> 2) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

// Swizzled K-major operands: a row of kc FP32 values is one row of the
// swizzle atom (32, 64 or 128 bytes: kc = 8, 16 or 32), 8 rows per atom,
// and the 16-byte chunk index within the row is XORed with bits of the row
// index (the address bits 4.. with the bits 7..; atoms start on multiples of
// their size).  Other kc use the layout without swizzle.
__host__ __device__ constexpr int sw_mode(int kc) { return kc == 8 ? 1 : kc == 16 ? 2 : kc == 32 ? 3 : 0; }
template <int KC>
__host__ __device__ __forceinline__ unsigned op_offset(int row, int k) {
    constexpr int mode = sw_mode(KC);
    if constexpr (mode == 0) {
        return cm_offset(row, k, KC);
    } else {
        constexpr int pitch = KC * 4;                       // bytes per row of the atom
        constexpr int shift = mode == 1 ? 2 : mode == 2 ? 1 : 0;  // row bits that meet address bit 7
        constexpr int mask = (1 << mode) - 1;               // chunk bits that are swizzled
        const int r7 = row & 7;
        const int chunk = (k >> 2) ^ ((r7 >> shift) & mask);
        return (unsigned)((row >> 3) * 8 * pitch + r7 * pitch + (chunk << 4) + ((k & 3) << 2));
    }
}
// descriptor of an operand with this layout, start at addr (a K step moves
// it by 32 bytes): stride offset 8 rows, layout type 6 / 4 / 2 (32, 64, 128
// byte swizzle) in bits 61-63; without swizzle the core-matrix offsets
template <int KC>
__device__ __forceinline__ uint64_t op_desc(unsigned addr) {
    constexpr int mode = sw_mode(KC);
    if constexpr (mode == 0) {
        return umma_desc(addr, 128, 32u * KC);
    } else {
        constexpr uint64_t layout = mode == 1 ? 6ull : mode == 2 ? 4ull : 2ull;
        return umma_desc(addr, 16, 8u * KC * 4) | (layout << 61);
    }
}

}  // namespace tk
