// Device helpers shared by the batched tick kernels (not part of the C ABI):
// inline-PTX wrappers of tcgen05 (tensor memory, MMA, commit, loads), TMA and
// L2-prefetch instructions, the shared-memory matrix descriptors of the
// spike-operand and weight layouts, and the storage helpers of the
// interleaved potential layout (fp16, int16 or int32 elements).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "ranc_ptx.cuh"

namespace ranc {

// ---------------------------------------------------------------------------
// tcgen05 / TMA wrappers (inline PTX)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptors, 128-byte swizzle, descriptor version 1.
// Weights (A): K-major, rows of 64 fp16 along K, 8-row groups 1024 bytes apart
// (stride byte offset; the leading byte offset is unused for this swizzle).
__device__ __forceinline__ uint64_t smem_desc_kmajor(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1u << 16;             // leading byte offset (unused)
    d |= (uint64_t)(1024u >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1u << 46;             // version
    d |= (uint64_t)2u << 61;             // 128-byte swizzle
    return d;
}

// Spike operand (B): MN-major, rows of 64 samples (128 bytes) per axon; the
// 8-axon groups of one 64-sample half form 1024-byte swizzle atoms.  The two
// sample halves are 1024 bytes apart (leading byte offset) and consecutive
// 8-axon groups 2048 bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(1024u >> 4) << 16;   // leading byte offset
    d |= (uint64_t)(2048u >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1u << 46;             // version
    d |= (uint64_t)2u << 61;             // 128-byte swizzle
    return d;
}

// Instruction descriptor: D fp32, A and B fp16, A K-major, B MN-major (bit 16),
// M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 16) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// The same MMA with the instruction descriptor in a register (any shape or
// operand major-ness the descriptor encodes), kinds f16 and f8f6f4.
__device__ __forceinline__ void mma_f16_id(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_f8f6f4_id(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                              uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// 32 x 32 bit-matrix transpose across a warp: on return lane j holds the word
// whose bit i is bit j of lane i's input word.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu : s == 2 ? 0x33333333u : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
        x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
    }
    return x;
}

__device__ __forceinline__ uint32_t valid_mask(int n_valid, int first) {
    const int k = n_valid - first;
    return k >= 32 ? 0xffffffffu : (k <= 0 ? 0u : ((1u << k) - 1u));
}

// For an fp32 holding an integer x with |x| < 2^22, adding 1.5 * 2^23 puts x
// in the low mantissa bits: the result's bit pattern is 0x4B400000 + x.  The
// caller subtracts the bias (folded into its leak constant).
__device__ __forceinline__ int f32_bits_minus_bias(uint32_t bits) {
    return __float_as_int(__uint_as_float(bits) + 12582912.0f);
}

// Potentials hf*16 .. hf*16+15 of one 32-sample unit held as 16-byte vectors.
template <typename VT, int kVecs>
__device__ __forceinline__ void unpack16(const uint4 (&q)[kVecs], int hf, int (&v)[16]) {
    if constexpr (sizeof(VT) == 2) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint4 u = q[hf * 2 + k];
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                v[8 * k + 2 * e] = (int)(int16_t)(w[e] & 0xFFFFu);
                v[8 * k + 2 * e + 1] = (int)w[e] >> 16;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint4 u = q[hf * 4 + k];
            v[4 * k] = (int)u.x;
            v[4 * k + 1] = (int)u.y;
            v[4 * k + 2] = (int)u.z;
            v[4 * k + 3] = (int)u.w;
        }
    }
}

// Writes potentials hf*16 .. hf*16+15 of one 32-sample unit: vector k of the
// unit sits 32 vectors (one per neuron of the warp) after vector k-1.
template <typename VT>
__device__ __forceinline__ void store16(uint4 *p, int hf, const int (&v)[16]) {
    if constexpr (sizeof(VT) == 2) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                w[e] = ((uint32_t)v[8 * k + 2 * e] & 0xFFFFu) | ((uint32_t)v[8 * k + 2 * e + 1] << 16);
            p[(hf * 2 + k) * 32] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            p[(hf * 4 + k) * 32] = make_uint4((uint32_t)v[4 * k], (uint32_t)v[4 * k + 1], (uint32_t)v[4 * k + 2],
                                              (uint32_t)v[4 * k + 3]);
    }
}

// Potential storage: integer value <-> stored element.
template <typename VT>
__device__ __forceinline__ VT v_from_int(int x) {
    if constexpr (std::is_same<VT, __half>::value) return __int2half_rn(x);
    else return (VT)x;
}
template <typename VT>
__device__ __forceinline__ int v_to_int(VT x) {
    if constexpr (std::is_same<VT, __half>::value) return __half2int_rn(x);
    else return (int)x;
}

// One 16-byte vector of potentials all equal to x (the reset value v0).
template <typename VT>
__device__ __forceinline__ uint4 v_splat(int x) {
    uint32_t w;
    if constexpr (sizeof(VT) == 2) {
        const VT e = v_from_int<VT>(x);
        w = (uint32_t)(*reinterpret_cast<const uint16_t *>(&e)) * 0x10001u;
    } else {
        w = (uint32_t)x;
    }
    return make_uint4(w, w, w, w);
}

// Deferred idle ticks of a lazy item: x <- max(x + pl, theta-) on every
// potential of a unit (pl = ticks * leak <= 0; the result lies in
// [theta-, x], so it is exact in every storage format).  pl is a 64-bit
// product: the up to 250 deferred ticks of an item times a leak near the int32 limit do not fit
// 32 bits, and x + pl is formed in 64 bits before the maximum.
template <typename VT, int kVecs>
__device__ __forceinline__ void defer_apply(uint4 (&q)[kVecs], long long pl, int nth) {
    // fp16 potentials and theta- lie within +-2048: any pl below -4096 gives
    // theta-, so the clamped value is exact in fp32.
    const float plf = (float)max(pl, -8192ll);
#pragma unroll
    for (int e = 0; e < kVecs; ++e) {
        uint32_t w[4] = {q[e].x, q[e].y, q[e].z, q[e].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if constexpr (std::is_same<VT, __half>::value) {
                const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
                const __half2 r = __floats2half2_rn(fmaxf(f.x + plf, (float)nth), fmaxf(f.y + plf, (float)nth));
                w[k] = *reinterpret_cast<const uint32_t *>(&r);
            } else if constexpr (sizeof(VT) == 2) {
                const int lo = (int)max((long long)(int16_t)(w[k] & 0xFFFFu) + pl, (long long)nth),
                          hi = (int)max((long long)((int)w[k] >> 16) + pl, (long long)nth);
                w[k] = ((uint32_t)lo & 0xFFFFu) | ((uint32_t)hi << 16);
            } else {
                w[k] = (uint32_t)(int)max((long long)(int)w[k] + pl, (long long)nth);
            }
        }
        q[e] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Element offset of potential (tile j, core c, neuron n, sample 32*cc + i) in
// the interleaved layout described at the top of this file.
template <typename VT>
__device__ __forceinline__ size_t v_index(int j, int c, int cc, int n, int i, int C, int N) {
    constexpr int E = 16 / (int)sizeof(VT);
    return ((((size_t)j * C + c) * 4 + cc) * N + (n & ~31)) * 32 + (size_t)((i / E) * 32 + (n & 31)) * E + (i % E);
}

}  // namespace ranc
