// Crossbar products for a batch of samples in three exact tensor-core
// formulations (include/ranc_xbar.h): the integration step of the neuron
// block, dV[b][c][n] = sum over active axons a of sample b connected to
// neuron n of core c of w[type(a)][n] (Sec. II; Alg. 1 neuron block), timed
// on the same inputs to choose the instruction of the batched path.
//
// One CTA (256 threads) per (core, group of 128-sample tiles): the core's
// A operand (folded fp16 weights, or the 0/1 crossbar in e4m3 / int8) is
// copied into shared memory once by the TMA engine (one bulk copy of its
// pre-arranged image) and reused for every tile of the group; per tile the
// spike bits of the 128 samples are staged, the B operand built (samples x
// axons, K-major), the product computed, and the epilogue turns it into dV.
//
//   F16_FOLDED   tcgen05.mma kind::f16, M = 128 neurons x N = 128 samples x
//                K = 16, fp32 accumulators in tensor memory (one per
//                128-neuron slice), dV read back with tcgen05.ld.
//   F8_PER_TYPE  axons sorted by type, each type's range padded to 32;
//                tcgen05.mma kind::f8f6f4 (e4m3 0/1 operands, K = 32), one
//                accumulator per type (4 x 128 columns) for one slice at a
//                time; dV = sum_k w[k][n] * count_k in int32.
//   I8_MMA_SYNC  the same sorted order and per-type counts with
//                mma.sync.m16n8k32.s32.s8.s8.s32 (warp-level, operands from
//                shared memory by ldmatrix); each warp owns 32 neurons x 32
//                samples at a time and folds every type's counts into dV.
// Shapes: axons a multiple of 64 up to 256, neurons 128 or 256, up to 4 types.

#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "ranc_internal.cuh"
#include "ranc_ptx.cuh"
#include "ranc_tc.cuh"
#include "ranc_xbar.h"

namespace ranc {
namespace {

constexpr int kXT = 256;           // threads per CTA
constexpr int kXS = 128;           // samples per tile
constexpr uint32_t kXBlk = 16384;  // 16 KB operand block
constexpr int kMaxAW = 8;          // axons <= 256
constexpr int kTilesPerCta = 8;

// Instruction descriptors: D fp32, A and B K-major, M = 128, N = 128; A and B
// fp16 (kind::f16) or e4m3 (kind::f8f6f4: type code 0 for both).
constexpr uint32_t kIdescKK = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

struct XArgs {
    int form, C, A, N, NH, KB, AW, KP, T, tiles_per_cta;
    const uint8_t *img;        // per core: A-operand image (img_bytes each)
    long long img_bytes;
    const int8_t *ktype;       // per core: type of each 32-wide step of the sorted order (-1: padding), [C][KP/32]
    const uint16_t *perm;      // per core: axon at each sorted position (0xFFFF: padding), [C][KP]
    const int16_t *w4;         // per core and neuron: weights of types 0..3, [C][N][4]
    const uint32_t *spikes;    // [B][AW]
    int *dv;                   // [B][C][N] or NULL
    long long *sums;           // [B][C] or NULL
    int *err;
};

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_s8(int (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                       uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Output of one (neuron n, sample m of the tile) value: dV itself (when dv is
// set) and its share of the digest sum_n (n % 8 + 1) * dV (returned; a
// 32-neuron share fits int32: |dV| <= 256 * 2047).
__device__ __forceinline__ int emit(const XArgs &a, int c, int b, int n, int v) {
    if (a.dv) a.dv[((size_t)b * a.C + c) * a.N + n] = v;
    return ((n & 7) + 1) * v;
}

// Sums each of x[0..15] over the 32 lanes by halving exchanges (16 shuffles);
// on return lane L holds the total of index 8 b4 + 4 b3 + 2 b2 + b1, b_i the
// bits of L (lanes L and L ^ 1 hold the same total).
__device__ __forceinline__ int lane_sums16(int (&x)[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = lane & 16;
        const int send = up ? x[i] : x[i + 8], keep = up ? x[i + 8] : x[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 8;
        const int send = up ? x[i] : x[i + 4], keep = up ? x[i + 4] : x[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 4;
        const int send = up ? x[i] : x[i + 2], keep = up ? x[i + 2] : x[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const int send = up ? x[0] : x[1], keep = up ? x[1] : x[0];
        x[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return x[0] + __shfl_xor_sync(0xffffffffu, x[0], 1);
}

__device__ __forceinline__ int lane_sum_index(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

__global__ void __launch_bounds__(kXT, 1) xbar_kernel(const __grid_constant__ XArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_img, bar_mma;
    __shared__ uint32_t tmem_sh;
    __shared__ uint32_t sp[kXS][kMaxAW];          // spike bits of the tile's samples
    __shared__ unsigned long long dsum[kXS];      // digest per sample of the tile
    __shared__ int ok_sh;

    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int c = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int AW = a.AW, N = a.N, KP = a.KP;
    const bool tc = a.form != RANC_XBAR_I8_MMA_SYNC;
    uint8_t *Asm = base;
    uint8_t *Bsm = Asm + ((a.img_bytes + 1023) & ~1023ll);
    // I8: rows of KP + 16 bytes (ldmatrix rows 16 bytes apart in bank space).
    const int rowb = KP + 16;
    uint16_t *perm_sm = reinterpret_cast<uint16_t *>(Bsm + (tc ? (size_t)(KP / (a.form == RANC_XBAR_F16_FOLDED ? 64 : 128)) * kXBlk
                                                              : (size_t)kXS * rowb));
    int8_t *kt_sm = reinterpret_cast<int8_t *>(perm_sm + KP);

    if (tid == 0) {
        mbar_init(&bar_img, 1);
        mbar_init(&bar_mma, 1);
        fence_mbar_init();
        ok_sh = 1;
    }
    const uint32_t tcols = a.form == RANC_XBAR_F16_FOLDED ? (a.NH == 2 ? 256u : 128u) : 512u;
    if (tc && warp == 0) tmem_alloc(&tmem_sh, tcols);
    if (a.form != RANC_XBAR_F16_FOLDED) {
        for (int i = tid; i < KP; i += kXT) perm_sm[i] = a.perm[(size_t)c * KP + i];
        for (int i = tid; i < KP / 32; i += kXT) kt_sm[i] = a.ktype[(size_t)c * (KP / 32) + i];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar_img, (uint32_t)a.img_bytes);
        bulk_g2s(Asm, a.img + (size_t)c * a.img_bytes, (uint32_t)a.img_bytes, &bar_img);
    }
    // Types present in this core (an absent type's accumulator is never written).
    int tmask = 0;
    if (a.form != RANC_XBAR_F16_FOLDED)
        for (int s = 0; s < KP / 32; ++s)
            if (kt_sm[s] >= 0) tmask |= 1 << kt_sm[s];
    bool img_ready = false, img_landed = false;
    int nmma = 0;  // phases of bar_mma
    const int t0 = blockIdx.y * a.tiles_per_cta, t1 = min(a.T, t0 + a.tiles_per_cta);
    for (int t = t0; t < t1; ++t) {
        // ---- stage the tile's spike bits, clear the digest
        for (int i = tid; i < kXS * AW; i += kXT) sp[i / AW][i % AW] = a.spikes[((size_t)t * kXS + i / AW) * AW + i % AW];
        if (tid < kXS) dsum[tid] = 0ull;
        __syncthreads();
        // ---- B operand: row m = sample m of the tile, K-major
        if (a.form == RANC_XBAR_F16_FOLDED) {
            // block kb: 64 axons x 128 samples fp16, 8 chunks of 16 bytes (8 axons) per row, chunk q at q ^ (m % 8)
            for (int i = tid; i < kXS * (a.A / 8); i += kXT) {
                const int m = i % kXS, g8 = i / kXS, kb = g8 >> 3, q = g8 & 7;
                const uint32_t by = (sp[m][g8 >> 2] >> ((g8 & 3) * 8)) & 0xFFu;
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    w[e] = (((by >> (2 * e)) & 1u) ? 0x3C00u : 0u) | (((by >> (2 * e + 1)) & 1u) ? 0x3C000000u : 0u);
                *reinterpret_cast<uint4 *>(Bsm + (size_t)kb * kXBlk + m * 128 + ((q ^ (m & 7)) << 4)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        } else {
            // 16 sorted positions per task; f8: block of 128 positions, chunk q at q ^ (m % 8); i8: plain rows
            const uint8_t one = a.form == RANC_XBAR_F8_PER_TYPE ? 0x38 : 0x01;  // e4m3 1.0 / int8 1
            for (int i = tid; i < kXS * (KP / 16); i += kXT) {
                const int m = i % kXS, g16 = i / kXS;
                uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int ax = perm_sm[g16 * 16 + e];
                    if (ax != 0xFFFF && ((sp[m][ax >> 5] >> (ax & 31)) & 1u)) w[e >> 2] |= (uint32_t)one << (8 * (e & 3));
                }
                uint8_t *dst = a.form == RANC_XBAR_F8_PER_TYPE
                                   ? Bsm + (size_t)(g16 >> 3) * kXBlk + m * 128 + (((g16 & 7) ^ (m & 7)) << 4)
                                   : Bsm + (size_t)m * rowb + g16 * 16;
                *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        if (tc) fence_async_smem();
        __syncthreads();
        if (!img_ready) {
            img_landed = mbar_wait_bounded(&bar_img, 0);
            if (!img_landed) {
                if (tid == 0) atomicExch(a.err, kErrTimeout);
                ok_sh = 0;
            }
            img_ready = true;
            __syncthreads();
            if (!ok_sh) break;
        }
        // ---- product and epilogue
        if (a.form == RANC_XBAR_F16_FOLDED) {
            if (tid == 0) {
                tc_fence_after();
                for (int h = 0; h < a.NH; ++h)
                    for (int kb = 0; kb < a.KB; ++kb)
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks)
                            mma_f16_id(tmem + h * 128, smem_desc_kmajor(smem_u32(Asm + (size_t)(h * a.KB + kb) * kXBlk) + ks * 32),
                                       smem_desc_kmajor(smem_u32(Bsm + (size_t)kb * kXBlk) + ks * 32), kIdescKK, (kb | ks) != 0);
                mma_commit(&bar_mma);
            }
            if (!mbar_wait_bounded(&bar_mma, nmma & 1) && lane == 0) atomicExch(a.err, kErrTimeout);
            ++nmma;
            tc_fence_after();
            // warp: lane quarter q (neurons 32q.. of each slice), 64-sample half ch
            const int q = warp & 3, ch = warp >> 2;
            for (int h = 0; h < a.NH; ++h) {
                const int n = h * 128 + q * 32 + lane;
#pragma unroll 1
                for (int cg = 0; cg < 4; ++cg) {
                    uint32_t d[16];
                    __syncwarp();
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 128 + ch * 64 + cg * 16), d);
                    int x[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        x[i] = emit(a, c, t * kXS + ch * 64 + cg * 16 + i, n, __float2int_rn(__uint_as_float(d[i])));
                    const int tot = lane_sums16(x, lane);
                    if (!(lane & 1)) atomicAdd(&dsum[ch * 64 + cg * 16 + lane_sum_index(lane)], (unsigned long long)(long long)tot);
                }
            }
        } else if (a.form == RANC_XBAR_F8_PER_TYPE) {
            const int q = warp & 3, ch = warp >> 2;
            for (int h = 0; h < a.NH; ++h) {
                if (tid == 0) {
                    tc_fence_after();
                    int prev = -1;
                    for (int s = 0; s < KP / 32; ++s) {
                        const int k = kt_sm[s];
                        if (k < 0) continue;
                        mma_f8f6f4_id(tmem + k * 128, smem_desc_kmajor(smem_u32(Asm + (size_t)(h * (KP / 128) + (s >> 2)) * kXBlk) + (s & 3) * 32),
                                      smem_desc_kmajor(smem_u32(Bsm + (size_t)(s >> 2) * kXBlk) + (s & 3) * 32), kIdescKK, k == prev);
                        prev = k;
                    }
                    mma_commit(&bar_mma);
                }
                if (!mbar_wait_bounded(&bar_mma, nmma & 1) && lane == 0) atomicExch(a.err, kErrTimeout);
                ++nmma;
                tc_fence_after();
                const int n = h * 128 + q * 32 + lane;
                const uint2 wq = *reinterpret_cast<const uint2 *>(a.w4 + ((size_t)c * N + n) * 4);
                const int wk[4] = {(int)(int16_t)(wq.x & 0xFFFFu), (int)wq.x >> 16, (int)(int16_t)(wq.y & 0xFFFFu), (int)wq.y >> 16};
#pragma unroll 1
                for (int cg = 0; cg < 4; ++cg) {
                    int v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (!((tmask >> k) & 1)) continue;
                        uint32_t d[16];
                        __syncwarp();
                        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(k * 128 + ch * 64 + cg * 16), d);
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] += wk[k] * __float2int_rn(__uint_as_float(d[i]));
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = emit(a, c, t * kXS + ch * 64 + cg * 16 + i, n, v[i]);
                    const int tot = lane_sums16(v, lane);
                    if (!(lane & 1)) atomicAdd(&dsum[ch * 64 + cg * 16 + lane_sum_index(lane)], (unsigned long long)(long long)tot);
                }
                tc_fence_before();
                __syncthreads();  // the next slice's MMAs write the same accumulators
            }
        } else {
            // I8: warp w owns neurons [32 (w % NW32), +32) and samples [64 (w / NW32) ...) in groups of 32.
            const int nw32 = N / 32, spw = kXS / (kXT / 32 / nw32);  // samples per warp
            const int nb0 = (warp % nw32) * 32, s_lo = (warp / nw32) * spw;
            const int g = lane >> 2, tq = lane & 3;
            int wk[2][2][4];  // [m16 tile][row half][type]
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const uint2 wq = *reinterpret_cast<const uint2 *>(a.w4 + ((size_t)c * N + nb0 + 16 * i + g + 8 * r) * 4);
                    wk[i][r][0] = (int)(int16_t)(wq.x & 0xFFFFu);
                    wk[i][r][1] = (int)wq.x >> 16;
                    wk[i][r][2] = (int)(int16_t)(wq.y & 0xFFFFu);
                    wk[i][r][3] = (int)wq.y >> 16;
                }
            const uint32_t a_base = smem_u32(Asm), b_base = smem_u32(Bsm);
            for (int s0 = s_lo; s0 < s_lo + spw; s0 += 32) {
                int dvr[2][4][4];
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int jn = 0; jn < 4; ++jn)
#pragma unroll
                        for (int e = 0; e < 4; ++e) dvr[i][jn][e] = 0;
                int s = 0;
                while (s < KP / 32) {
                    const int k = kt_sm[s];
                    if (k < 0) {
                        ++s;
                        continue;
                    }
                    int acc[2][4][4];
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int jn = 0; jn < 4; ++jn)
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[i][jn][e] = 0;
                    for (; s < KP / 32 && kt_sm[s] == k; ++s) {
                        const int k0 = s * 32;
                        uint32_t af[2][4], bf[4][2];
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const int row = nb0 + 16 * i + (lane & 7) + 8 * ((lane >> 3) & 1);
                            ldsm_x4(a_base + row * rowb + k0 + 16 * (lane >> 4), af[i][0], af[i][1], af[i][2], af[i][3]);
                        }
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            const int smp = s0 + 16 * p + (lane & 7) + 8 * (lane >> 4);
                            ldsm_x4(b_base + smp * rowb + k0 + 16 * ((lane >> 3) & 1), bf[2 * p][0], bf[2 * p][1], bf[2 * p + 1][0],
                                    bf[2 * p + 1][1]);
                        }
#pragma unroll
                        for (int i = 0; i < 2; ++i)
#pragma unroll
                            for (int jn = 0; jn < 4; ++jn)
                                mma_s8(acc[i][jn], af[i][0], af[i][1], af[i][2], af[i][3], bf[jn][0], bf[jn][1]);
                    }
                    int wc[2][2];  // this type's weight of the thread's four neurons (selects: k is not a constant)
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int r = 0; r < 2; ++r)
                            wc[i][r] = k == 0 ? wk[i][r][0] : k == 1 ? wk[i][r][1] : k == 2 ? wk[i][r][2] : wk[i][r][3];
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int jn = 0; jn < 4; ++jn)
#pragma unroll
                            for (int e = 0; e < 4; ++e) dvr[i][jn][e] += wc[i][e >> 1] * acc[i][jn][e];
                }
                // fragment element e of tile (i, jn): neuron nb0 + 16i + g + 8 (e / 2), sample s0 + 8 jn + 2 tq + e % 2
#pragma unroll
                for (int jn = 0; jn < 4; ++jn)
#pragma unroll
                    for (int e1 = 0; e1 < 2; ++e1) {
                        const int m = s0 + 8 * jn + 2 * tq + e1;
                        int sm = 0;
#pragma unroll
                        for (int i = 0; i < 2; ++i)
#pragma unroll
                            for (int r = 0; r < 2; ++r)
                                sm += emit(a, c, t * kXS + m, nb0 + 16 * i + g + 8 * r, dvr[i][jn][2 * r + e1]);
                        // lanes with the same tq hold the same samples: reduce over g
#pragma unroll
                        for (int o = 4; o < 32; o <<= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
                        if (g == 0) atomicAdd(&dsum[m], (unsigned long long)(long long)sm);
                    }
            }
        }
        if (tc) tc_fence_before();
        __syncthreads();
        if (a.sums && tid < kXS) a.sums[((size_t)t * kXS + tid) * a.C + c] = (long long)dsum[tid];
    }
    if (!img_landed && tid == 0) mbar_wait_bounded(&bar_img, 0);  // the copy lands before the CTA exits
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tc && warp == 0) tmem_dealloc(tmem, tcols);
}

}  // namespace
}  // namespace ranc

using namespace ranc;

struct ranc_xbar {
    int form = 0, C = 0, A = 0, N = 0, NH = 0, KB = 0, KP = 0, device = 0;
    long long img_bytes = 0;
    size_t smem = 0;
    cudaStream_t stream = nullptr;
    uint8_t *img = nullptr;
    int8_t *ktype = nullptr;
    uint16_t *perm = nullptr;
    int16_t *w4 = nullptr;
    int *err = nullptr;
    std::string last_error;
};

namespace {
thread_local std::string g_xbar_create_error;

int xfail(ranc_xbar *x, int code, const char *fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    (x ? x->last_error : g_xbar_create_error) = buf;
    return code;
}

void xfree(ranc_xbar *x) {
    void *ptrs[] = {x->img, x->ktype, x->perm, x->w4, x->err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}
}  // namespace

extern "C" int ranc_xbar_create(const ranc_desc *d, int32_t form, void *cuda_stream, ranc_xbar **out) {
    if (!out) return xfail(nullptr, RANC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d || !d->crossbar || !d->axon_type || !d->weight) return xfail(nullptr, RANC_EINVAL, "incomplete description");
    const int C = d->n_cores, A = d->axons, N = d->neurons, K = d->n_types;
    if (form < RANC_XBAR_F16_FOLDED || form > RANC_XBAR_I8_MMA_SYNC) return xfail(nullptr, RANC_EINVAL, "unknown form %d", form);
    if (C < 1 || A % 64 || A < 64 || A > 256 || (N != 128 && N != 256) || K < 1 || K > 4)
        return xfail(nullptr, RANC_EINVAL, "the crossbar kernels need axons a multiple of 64 in [64, 256], neurons 128 or "
                                           "256 and 1..4 axon types");
    for (size_t i = 0; i < (size_t)C * A; i++)
        if (d->axon_type[i] >= K) return xfail(nullptr, RANC_EINVAL, "axon type out of range");
    for (size_t i = 0; i < (size_t)C * K * N; i++)
        if (d->weight[i] > 2047 || d->weight[i] < -2047) return xfail(nullptr, RANC_EINVAL, "|weight| > 2047");
    ranc_xbar *x = new (std::nothrow) ranc_xbar();
    if (!x) return xfail(nullptr, RANC_ENOMEM, "host allocation");
    x->form = form; x->C = C; x->A = A; x->N = N; x->NH = N / 128; x->KB = A / 64;
    x->stream = static_cast<cudaStream_t>(cuda_stream);
    auto abort_create = [&](int code, const char *msg) {
        g_xbar_create_error = msg;
        xfree(x);
        delete x;
        return code;
    };
    cudaError_t e = cudaGetDevice(&x->device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, x->device);
    if (e != cudaSuccess) return abort_create(RANC_ECUDA, "no CUDA device");
    if (prop.major != 10 || prop.minor != 3) return abort_create(RANC_EINVAL, "the crossbar kernels need an sm_103 (GB300) device");
    const int NWd = N / 32;
    auto conn = [&](int c, int ax, int n) { return (d->crossbar[((size_t)c * A + ax) * NWd + (n >> 5)] >> (n & 31)) & 1u; };
    // Type-sorted order (per-type forms): each type's positions padded to 32;
    // the total padded to 128 (e4m3 blocks), the same for every core.
    int KP = A;
    std::vector<std::vector<int>> order(C);
    std::vector<int8_t> kt;
    if (form != RANC_XBAR_F16_FOLDED) {
        int kp_max = 0;
        for (int c = 0; c < C; c++) {
            int p = 0;
            for (int k = 0; k < K; k++) {
                int nk = 0;
                for (int ax = 0; ax < A; ax++)
                    if (d->axon_type[(size_t)c * A + ax] == k) ++nk;
                p += (nk + 31) / 32 * 32;
            }
            kp_max = std::max(kp_max, p);
        }
        KP = (kp_max + 127) / 128 * 128;
        kt.assign((size_t)C * (KP / 32), (int8_t)-1);
        for (int c = 0; c < C; c++) {
            order[c].assign(KP, 0xFFFF);
            int p = 0;
            for (int k = 0; k < K; k++) {
                const int p0 = p;
                for (int ax = 0; ax < A; ax++)
                    if (d->axon_type[(size_t)c * A + ax] == k) order[c][p++] = ax;
                p = (p + 31) / 32 * 32;
                for (int s = p0 / 32; s < p / 32; s++) kt[(size_t)c * (KP / 32) + s] = (int8_t)k;
            }
        }
    }
    x->KP = KP;
    // A-operand image of every core.
    size_t img_bytes;
    if (form == RANC_XBAR_F16_FOLDED) img_bytes = (size_t)x->NH * x->KB * kXBlk;
    else if (form == RANC_XBAR_F8_PER_TYPE) img_bytes = (size_t)x->NH * (KP / 128) * kXBlk;
    else img_bytes = (size_t)N * (KP + 16);
    x->img_bytes = (long long)img_bytes;
    std::vector<uint8_t> img(img_bytes * C, 0);
    std::vector<int16_t> w4((size_t)C * N * 4, 0);
    std::vector<uint16_t> perm((size_t)C * KP, 0xFFFF);
    for (int c = 0; c < C; c++) {
        uint8_t *im = img.data() + img_bytes * c;
        for (int n = 0; n < N; n++)
            for (int k = 0; k < K; k++) w4[((size_t)c * N + n) * 4 + k] = d->weight[((size_t)c * K + k) * N + n];
        if (form == RANC_XBAR_F16_FOLDED) {
            // block (h, kb): row r = neuron 128h + r, 64 fp16 of axons 64kb.., chunk q at q ^ (r % 8)
            for (int ax = 0; ax < A; ax++) {
                const int k = d->axon_type[(size_t)c * A + ax], kb = ax >> 6, q = (ax & 63) >> 3, e8 = ax & 7;
                for (int n = 0; n < N; n++) {
                    if (!conn(c, ax, n)) continue;
                    const int h = n >> 7, r = n & 127;
                    const __half hv = __float2half((float)d->weight[((size_t)c * K + k) * N + n]);
                    uint16_t *row = reinterpret_cast<uint16_t *>(im + (size_t)(h * x->KB + kb) * kXBlk + r * 128);
                    row[((q ^ (r & 7)) << 3) + e8] = *reinterpret_cast<const uint16_t *>(&hv);
                }
            }
        } else {
            for (int p = 0; p < KP; p++) {
                const int ax = order[c][p];
                perm[(size_t)c * KP + p] = (uint16_t)ax;
                if (ax == 0xFFFF) continue;
                for (int n = 0; n < N; n++) {
                    if (!conn(c, ax, n)) continue;
                    if (form == RANC_XBAR_F8_PER_TYPE) {  // block (h, p / 128): row n % 128, chunk (p % 128) / 16 swizzled
                        const int h = n >> 7, r = n & 127, q = (p & 127) >> 4;
                        im[(size_t)(h * (KP / 128) + (p >> 7)) * kXBlk + r * 128 + ((q ^ (r & 7)) << 4) + (p & 15)] = 0x38;
                    } else {
                        im[(size_t)n * (KP + 16) + p] = 1;
                    }
                }
            }
        }
    }
    if (dev_alloc((void **)&x->img, img.size()) != cudaSuccess || dev_alloc((void **)&x->w4, w4.size() * 2) != cudaSuccess ||
        dev_alloc((void **)&x->perm, perm.size() * 2) != cudaSuccess ||
        dev_alloc((void **)&x->ktype, std::max<size_t>(kt.size(), 1)) != cudaSuccess ||
        dev_alloc((void **)&x->err, 4) != cudaSuccess)
        return abort_create(RANC_ENOMEM, "device allocation of the crossbar images");
    if (cudaMemcpy(x->img, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(x->w4, w4.data(), w4.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(x->perm, perm.data(), perm.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        (!kt.empty() && cudaMemcpy(x->ktype, kt.data(), kt.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemset(x->err, 0, 4) != cudaSuccess)
        return abort_create(RANC_ECUDA, "copy of the crossbar images");
    const size_t bbytes = form == RANC_XBAR_F16_FOLDED ? (size_t)x->KB * kXBlk
                          : form == RANC_XBAR_F8_PER_TYPE ? (size_t)(KP / 128) * kXBlk
                                                          : (size_t)kXS * (KP + 16);
    x->smem = 1024 + ((img_bytes + 1023) & ~(size_t)1023) + bbytes + (size_t)KP * 2 + KP / 32 + 16;
    if (x->smem > 227 * 1024 - 8192) return abort_create(RANC_EINVAL, "the operands of this shape do not fit shared memory");
    if (raise_smem_limit((const void *)xbar_kernel, (int)x->smem) != cudaSuccess)
        return abort_create(RANC_ECUDA, "kernel shared-memory attribute");
    *out = x;
    return RANC_OK;
}

extern "C" int ranc_xbar_run(ranc_xbar *x, const uint32_t *spikes, int32_t batch, int32_t *dv, int64_t *sums) {
    if (!x) return RANC_EINVAL;
    if (!spikes || batch < 0 || batch % kXS) return xfail(x, RANC_EINVAL, "spikes NULL or batch not a multiple of 128");
    if (batch == 0) return RANC_OK;
    XArgs a{};
    a.form = x->form; a.C = x->C; a.A = x->A; a.N = x->N; a.NH = x->NH; a.KB = x->KB; a.AW = x->A / 32; a.KP = x->KP;
    a.T = batch / kXS; a.tiles_per_cta = kTilesPerCta; a.img = x->img; a.img_bytes = x->img_bytes; a.ktype = x->ktype;
    a.perm = x->perm; a.w4 = x->w4; a.spikes = spikes; a.dv = dv; a.sums = reinterpret_cast<long long *>(sums); a.err = x->err;
    const dim3 grid(x->C, (a.T + kTilesPerCta - 1) / kTilesPerCta);
    xbar_kernel<<<grid, kXT, x->smem, x->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return xfail(x, RANC_ECUDA, "crossbar kernel launch: %s", cudaGetErrorString(e));
    return RANC_OK;
}

extern "C" int ranc_xbar_sync(ranc_xbar *x) {
    if (!x) return RANC_EINVAL;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, x->err, 4, cudaMemcpyDeviceToHost, x->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
    if (e != cudaSuccess) return xfail(x, RANC_ECUDA, "crossbar kernel: %s", cudaGetErrorString(e));
    if (h == kErrTimeout) return xfail(x, RANC_ETIMEOUT, "a device-side wait gave up");
    return RANC_OK;
}

extern "C" void ranc_xbar_destroy(ranc_xbar *x) {
    if (!x) return;
    cudaStreamSynchronize(x->stream);
    xfree(x);
    delete x;
}

extern "C" const char *ranc_xbar_last_error(const ranc_xbar *x) {
    return x ? x->last_error.c_str() : g_xbar_create_error.c_str();
}
