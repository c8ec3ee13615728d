// Batched path: 128 samples per tile, crossbar integration on the
// 5th-generation tensor cores (tcgen05), one persistent launch per tick.
//
// Per (core c, sample tile j) work item, one tick of Alg. 1:
//   dV[n][m] = sum_a W[n][a] * S[m][a]            (Sec. II, Alg. 1 neuron block)
// where S[m][a] in {0, 1} is "axon a of sample m is active" and
// W[n][a] = w[type(a)][n] if axon a connects to neuron n, else 0 (the weight
// chosen by axon type, folded into the connection matrix once at create).
// Both operands are exact in fp16 (|w| <= 2047) and every partial sum is an
// integer below 2^22 in magnitude, so fp32 accumulation in tensor memory is
// exact and the result equals the integer sum of the CPU definition.
//
// Roles inside one CTA (640 threads, one CTA per SM, persistent over items):
//   all         the split (split_items): every item of the tick is classified
//               active / idle / lazy (see item_class) and the CTA takes its
//               share of the items by a cost prefix computed in every CTA;
//   warps 0-15  workers (104 registers after setmaxnreg).  Iteration i over
//               the CTA's items that are not lazy: (1) read and clear the
//               scheduler row of tick t for item i (loaded one build ahead)
//               and expand its bits to the fp16 0/1 operand S
//               (sample-contiguous, 128-byte swizzled: a scheduler word is
//               already 32 consecutive samples of one axon, so no transpose;
//               zero for an idle item); (2) epilogue of item i-1 while the
//               tensor core works on item i: tensor memory -> registers
//               (tcgen05.ld), potential update (leak, thresholds, reset),
//               spike masks over 32 samples per neuron, delivery of a
//               neuron's spike masks with one atomicOr into the sample-minor
//               scheduler rows (and the destination row's stamp), output-bus
//               counts;
//   warps 16-19 one warpgroup (48 registers after setmaxnreg); warp 16:
//               tensor-memory allocation, TMA loads of the folded weights of
//               the current core (cp.async.bulk.tensor, 128-byte swizzle),
//               L2 prefetch of the next items' potentials and rows,
//               tcgen05.mma issue and commit.
// Every mbarrier wait is bounded (global timer); a timeout sets the device
// error word and all roles leave their loops, drain the tensor core and free
// tensor memory before the CTA exits.
//
// Layouts (T tiles of 128 samples; sample m of tile j is batch index 128j+m):
//   V     [T][C][4][N/32][P][32][E]  potentials (fp16, int16 or int32, the
//                                    narrowest that is exact for the network):
//                                    for 32-sample chunk cc and
//                                    neuron group n/32, piece p holds samples
//                                    E*p .. E*p+E-1 of the 32 neurons side by
//                                    side (E = 16 bytes / element size, P = 32 / E),
//                                    so a warp's 16-byte accesses are contiguous
//   ring  [T][C][16][A][4]   scheduler rows: word k of axon a holds samples 32k..32k+31
//   spk   [T][C][4][N]       spike masks of the last tick (32 samples per word)
//   inT   [T][ticks][Lpad][4] input lines, same sample-minor packing
//   stamp [16][items]        per scheduler row and item (item it = c*T + j): the
//                            cycle of the tick that reads the row, written on delivery
//   pend  [2][items]         deferred idle ticks per item (by tick parity)

#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "ranc_internal.cuh"
#include "ranc_ptx.cuh"
#include "ranc_tc.cuh"

namespace ranc {
namespace {

constexpr int kWorkers = 16;                 // warps 0-15: operand build + epilogue
constexpr int kMmaWarp = 16;                 // warp 16: TMEM, TMA, MMA issue
constexpr int kThreads = (kWorkers + 4) * 32;  // warps 16-19: one warpgroup, warp 16 issues the MMAs
// Registers per thread after the prologue: the issuer's warpgroup gives up
// registers that the workers take (setmaxnreg).  The launch provides
// kThreads * 96 = 61440; 16 * 32 * kRegWorker + 4 * 32 * kRegIssuer = 59392
// (per SM sub-partition: 4 worker warps and 1 issuer-group warp, 14848 of 16384).
constexpr int kRegWorker = 104, kRegIssuer = 48;
static_assert(kWorkers * 32 * kRegWorker + 4 * 32 * kRegIssuer <= kThreads * 96, "register split exceeds the launch");
constexpr uint32_t kBlockBytes = 128u * 128u;  // one 64-axon K-block: 128 weight rows or 128 samples x 64 fp16
constexpr int kClsCap = 16384;                 // items of a CTA whose classes are kept in shared memory

struct TickArgs {
    int C, A, N, NH, KB, T, n_valid, Lpad, in_ticks, n_out, neg_mode, items;
    long long tick;
    const int4 *prm;
    const uint2 *dst;
    const int *fin_ptr, *fin_line;
    const uint32_t *outdeg;  // [C][A] connections of each axon
    const uint4 *inT;
    const int *v0;           // non-NULL: the potentials are still the reset values v0 [C][N] (V is not read)
    void *V;
    uint4 *ring;
    uint32_t *spk, *out;
    unsigned long long *cnt;
    int *err;
    uint32_t tmem_cols;
    uint32_t *olog;          // NULL, or this tick's output-bus log: sample b < olog_rows, id -> olog[b * olog_stride + id]
    long long olog_stride;
    int olog_rows;
    // Item activity (see item_class).  Item it = c * T + j.
    const uint8_t *stamp_row;  // [items] stamps of this tick's scheduler row
    uint8_t *stamp;            // [16][spitch]: a delivery into row r of item it writes stamp[r][it] = its cycle
    long long spitch;
    uint32_t sclock;           // stamp clock of this tick (== tick mod 16); its cycle is (sclock >> 4) mod 256
    int all_active;            // every row may hold bits (imported state): no item is idle
    const uint8_t *core_flags; // [C] bit 0: some input line drives the core; bit 1: its idle ticks can be deferred;
                               // bit 2: some neuron of the core sends its spikes to the output bus
    const uint8_t *pend_in;    // [items] idle ticks deferred before this tick
    uint8_t *pend_out;         // [items] idle ticks deferred after this tick
    int cost_active, cost_idle, cost_lazy, cost_wake, cost_out;  // relative costs for the split of the items over the CTAs
    unsigned long long *item_ticks;  // [3]: items updated, items whose tick was deferred, active items (accumulated)
    int stall_test;            // failure-detection tests only: CTA 0 waits for a weight copy on a barrier
                               // armed with a transaction count that no copy satisfies
    int dbg_plant;             // debug builds: site whose range checks fail on purpose (0: none)
};

constexpr int kPendMax = 250;  // deferred idle ticks of an item are applied before this many accumulate

// Work classes of an item in one tick.
//   2 active: its scheduler row may hold bits, or input lines drive its core
//     in this tick: full update (operand build, MMA, epilogue).
//   1 idle: no synaptic input: no row or input is read, the operand is zero
//     and only its first K-step is issued (dV = W * 0 = 0), so the item takes
//     the same epilogue as an active one.
//   0 lazy: idle, and the core's idle tick is a deferred map (every neuron has
//     leak <= 0, theta- < theta+, reset < theta+, v0 < theta+, saturating
//     negative threshold): no potential is stored at or above theta+, so with
//     dV = 0 nothing fires and V <- max(V + leak, theta-); k such ticks compose
//     to V <- max(V + k * leak, theta-).  The item only counts the tick; the
//     count is applied by the next update that reads V (or before a state
//     read).  Never in the first tick after a reset (V is v0 and unwritten).
// A row holds bits only after a delivery into it, and every delivery writes
// the row's stamp with the cycle of the tick that will read it, so an item
// whose stamp differs has an empty row.  An equal stamp left over from an
// earlier cycle only makes an empty item "active", which is still exact.
// The class from the item's stamp, deferred ticks and core flags.
__device__ __forceinline__ int class_from(const TickArgs &a, uint8_t stamp, uint8_t pend, uint8_t cflags) {
    if (a.all_active || stamp == (uint8_t)(a.sclock >> 4) || (a.tick < (long long)a.in_ticks && (cflags & 1)))
        return 2;
    if (!a.v0 && (cflags & 2) && pend < kPendMax) return 0;
    return 1;
}
__device__ __forceinline__ int item_class(const TickArgs &a, int it) {
    return class_from(a, a.stamp_row[it], a.pend_in[it], a.core_flags[it / a.T]);
}


// ---------------------------------------------------------------------------
// The tick kernel
// ---------------------------------------------------------------------------

// Split of one tick's items over the CTAs, run by every thread of a CTA at
// kernel start (kept out of line so that it does not weigh on the register
// allocation of the item loop).  CTA b takes the items whose cost prefix P
// (exclusive, in item order) satisfies b * W <= P * G < (b + 1) * W, W the
// total cost and G the grid; every CTA computes the same sums.  On return
// cut_sh holds this CTA's range [i0, i1); when the range fits kClsCap, cls_sm
// holds the class of each of its items (bit 2: deferred idle ticks before
// this tick); pend_out holds the deferred ticks after this tick of each of its
// items; flags_sh bit 0 is set when some item applies deferred ticks in this
// tick; bit k of nl_bits[0] is set when item i0 + k is not lazy, of
// nl_bits[1] when it applies deferred ticks.  A range that does not fit
// kClsCap defers nothing: its lazy items are updated as idle ones (and only
// flags_sh and pend_out are written).  A lazy item's spike masks are left as
// they are: its last tick fired nothing, and the pass that applies deferred
// ticks before a state read clears them.
__device__ __noinline__ void split_items(const TickArgs &a, long long *wsum_sh, int *cut_sh, uint8_t *cls_sm,
                                         int *flags_sh, uint32_t (*nl_bits)[kClsCap / 32]) {
    // The arguments this function reads, once (a reference to the kernel's
    // argument block is a generic pointer here: every field read would be a load).
    const uint8_t *const stamp_row = a.stamp_row, *const pend_in = a.pend_in, *const core_flags = a.core_flags;
    uint8_t *const pend_out = a.pend_out;
    unsigned long long *const item_ticks = a.item_ticks;
    const int items = a.items, T = a.T;
    const bool all_active = a.all_active != 0, first = a.v0 != nullptr, inputs = a.tick < (long long)a.in_ticks;
    const uint8_t cycle = (uint8_t)(a.sclock >> 4);
    const int c_act = a.cost_active, c_idle = a.cost_idle, c_lazy = a.cost_lazy, c_wake = a.cost_wake, c_out = a.cost_out;
    // As class_from, on those copies.
    auto cls_from = [&](uint8_t stamp, uint8_t pend, uint8_t cflags) -> int {
        if (all_active || stamp == cycle || (inputs && (cflags & 1))) return 2;
        if (!first && (cflags & 2) && pend < kPendMax) return 0;
        return 1;
    };
    // Thread tid classifies items [tid * per, tid * per + per), a multiple of
    // 16, reading stamps and deferred counts as 16-byte vectors (rows are
    // padded to 128 bytes).
    const int per = ((items + kThreads - 1) / kThreads + 15) & ~15;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t0 = min(items, tid * per), t1 = min(items, t0 + per);
    for (int w = tid; w < 2 * kClsCap / 32; w += kThreads) nl_bits[w / (kClsCap / 32)][w % (kClsCap / 32)] = 0u;
    // fn(it, class, deferred idle ticks, core flags) for the items [u0, u1) of this thread.
    auto visit = [&](int u0, int u1, auto &&fn) {
        if (u0 >= u1) return;
        int c = u0 / T, j = u0 - c * T;
        uint8_t cf = core_flags[c];
        uint4 sv = *reinterpret_cast<const uint4 *>(stamp_row + (u0 & ~15));
        uint4 pv = *reinterpret_cast<const uint4 *>(pend_in + (u0 & ~15));
        for (int b16 = u0 & ~15; b16 < u1; b16 += 16) {
            const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w}, pw[4] = {pv.x, pv.y, pv.z, pv.w};
            if (b16 + 16 < u1) {  // the next group's vectors are in flight while this one is classified
                sv = *reinterpret_cast<const uint4 *>(stamp_row + b16 + 16);
                pv = *reinterpret_cast<const uint4 *>(pend_in + b16 + 16);
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int it = b16 + k;
                if (it < u0) continue;
                if (it >= u1) break;
                if (j == T) {
                    j = 0;
                    cf = core_flags[++c];
                }
                ++j;
                const uint8_t pn = (uint8_t)(pw[k >> 2] >> (8 * (k & 3)));
                fn(it, cls_from((uint8_t)(sw[k >> 2] >> (8 * (k & 3))), pn, cf), first ? 0 : (int)pn, cf);
            }
        }
    };
    // Cost of an item: its class, plus the pass that applies deferred ticks
    // when it wakes up, plus the output-bus events of an updated item of an
    // output core.
    auto cost_of = [&](int cls, int pend, uint8_t cf) -> int {
        return (cls == 2 ? c_act : cls == 1 ? c_idle : c_lazy) + (cls != 0 && pend ? c_wake : 0) + (cls != 0 && (cf & 4) ? c_out : 0);
    };
    // Total cost of this thread's items.  A group of 16 items inside one core
    // is classified four at a time (bytes of the stamp and deferral vectors,
    // SIMD compares, class counts by popcount); other groups item by item.
    long long csum = 0;
    {
        const uint32_t cyc4 = cycle * 0x01010101u, lim4 = (uint32_t)kPendMax * 0x01010101u;
        for (int b16 = t0; b16 < t1; b16 += 16) {
            const int c = b16 / T;
            if (b16 + 16 > t1 || (b16 + 15) / T != c) {
                visit(b16, min(b16 + 16, t1), [&](int, int cls, int pend, uint8_t cf) { csum += cost_of(cls, pend, cf); });
                continue;
            }
            const uint4 sv = *reinterpret_cast<const uint4 *>(stamp_row + b16);
            const uint4 pv = *reinterpret_cast<const uint4 *>(pend_in + b16);
            const uint8_t cf = core_flags[c];
            const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w}, pw[4] = {pv.x, pv.y, pv.z, pv.w};
            const bool act_all = all_active || (inputs && (cf & 1)), lazy_ok = !first && (cf & 2);
            int n_act = 0, n_idle = 0, n_lazy = 0, n_wake = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // byte masks: 0xFF where the item is in the class
                const uint32_t ma = act_all ? 0xFFFFFFFFu : __vcmpeq4(sw[q], cyc4);
                const uint32_t mp = first ? 0u : __vcmpne4(pw[q], 0u);
                const uint32_t ml = lazy_ok ? ~ma & __vcmpltu4(pw[q], lim4) : 0u;
                const uint32_t mi = ~ma & ~ml;
                n_act += __popc(ma) >> 3;
                n_lazy += __popc(ml) >> 3;
                n_idle += __popc(mi) >> 3;
                n_wake += __popc(~ml & mp) >> 3;
            }
            csum += (long long)c_act * n_act + (long long)c_idle * n_idle + (long long)c_lazy * n_lazy +
                    (long long)c_wake * n_wake + ((cf & 4) ? (long long)c_out * (n_act + n_idle) : 0);
        }
    }
    long long cinc = csum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, cinc, o);
        if (lane >= o) cinc += y;
    }
    if (lane == 31) wsum_sh[warp] = cinc;
    __syncthreads();
    {
        long long P = 0, W = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            const long long x = wsum_sh[w];
            if (w < warp) P += x;
            W += x;
        }
        P += cinc - csum;
        // P * G < b * W  <=>  P < ceil(b * W / G): the first item of CTA b is
        // the first whose prefix reaches that bound.
        const long long G = gridDim.x;
        const long long lo = ((long long)blockIdx.x * W + G - 1) / G, hi = ((long long)(blockIdx.x + 1) * W + G - 1) / G;
        // Items of this thread whose prefix lies below a bound: all of them,
        // none, or (for at most one thread per bound) a walk.
        int n0 = 0, n1 = 0;
        const long long Pend = P + csum;
        const bool walk0 = P < lo && Pend > lo, walk1 = P < hi && Pend > hi;
        if (!walk0) n0 = Pend <= lo ? t1 - t0 : 0;
        if (!walk1) n1 = Pend <= hi ? t1 - t0 : 0;
        if (walk0 || walk1)
            visit(t0, t1, [&](int, int cls, int pend, uint8_t cf) {
                if (walk0) n0 += P < lo;
                if (walk1) n1 += P < hi;
                P += cost_of(cls, pend, cf);
            });
        n0 = __reduce_add_sync(0xffffffffu, n0);
        n1 = __reduce_add_sync(0xffffffffu, n1);
        if (lane == 0 && (n0 | n1)) {
            atomicAdd(&cut_sh[0], n0);
            atomicAdd(&cut_sh[1], n1);
        }
    }
    __syncthreads();
    const int i0 = cut_sh[0], i1 = cut_sh[1];
    const bool cls_cached = i1 - i0 <= kClsCap;
    int fl = 0, n_up = 0, n_def = 0, n_act = 0;
    visit(max(t0, i0), min(t1, i1), [&](int it, int cls, int pend, uint8_t) {
        if (!cls_cached && cls == 0) cls = 1;
        ++(cls != 0 ? n_up : n_def);
        n_act += cls == 2;
        if (cls_cached) {
            const int k = it - i0;
            cls_sm[k] = (uint8_t)(cls | (pend ? 4 : 0));
            if (cls != 0) atomicOr(&nl_bits[0][k >> 5], 1u << (k & 31));
            if (cls != 0 && pend) atomicOr(&nl_bits[1][k >> 5], 1u << (k & 31));
        }
        fl |= pend && cls != 0 ? 1 : 0;
        pend_out[it] = cls == 0 ? (uint8_t)(pend + 1) : (uint8_t)0;
    });
    if (fl) atomicOr(flags_sh, fl);
    n_up = __reduce_add_sync(0xffffffffu, n_up);
    n_def = __reduce_add_sync(0xffffffffu, n_def);
    if (lane == 0 && n_up) atomicAdd(item_ticks, (unsigned long long)n_up);
    if (lane == 0 && n_def) atomicAdd(item_ticks + 1, (unsigned long long)n_def);
    n_act = __reduce_add_sync(0xffffffffu, n_act);
    if (lane == 0 && n_act) atomicAdd(item_ticks + 2, (unsigned long long)n_act);
}

template <typename VT, int kNegReset>
__global__ void __launch_bounds__(kThreads, 1) batched_tick_kernel(const __grid_constant__ TickArgs a, const __grid_constant__ CUtensorMap wmap) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_w, bar_drain, s_full, s_free, acc_full[2], acc_empty[2], bar_stall;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ long long wsum_sh[kThreads / 32];
    __shared__ int cut_sh[2];
    __shared__ uint32_t nl_sh[2][kClsCap / 32];  // bit k: item i0 + k is not lazy / wakes up
    __shared__ int flags_sh;  // bit 0: some item applies deferred idle ticks

    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NH = a.NH, KB = a.KB, C = a.C, A = a.A, N = a.N, T = a.T;
    uint8_t *Wsm = base;                                   // [NH][KB] blocks of 128 rows x 128 B
    uint8_t *Ssm = Wsm + (size_t)NH * KB * kBlockBytes;    // [KB] blocks of [8 groups][2 halves][8 axons][64 samples]
    uint2 *lut = reinterpret_cast<uint2 *>(Ssm + (size_t)KB * kBlockBytes);  // 16 x 8 B: one row of banks
    // Per item of this CTA: class (bits 0-1) and "has deferred idle ticks" (bit 2).
    uint8_t *cls_sm = reinterpret_cast<uint8_t *>(lut) + 4096;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = (int)(a.tick & (kRows - 1));

    // 4 fp16 values (1.0 or 0.0) for every nibble of spike bits.  The table is
    // 128 bytes, so distinct entries sit in distinct banks and a warp's
    // lookups never conflict.
    if (tid < 16) {
        uint32_t w[2];
#pragma unroll
        for (int q = 0; q < 2; ++q)
            w[q] = (((tid >> (2 * q)) & 1) ? 0x3C00u : 0u) | (((tid >> (2 * q + 1)) & 1) ? 0x3C000000u : 0u);
        lut[tid] = make_uint2(w[0], w[1]);
    }
    if (tid == 0) {
        mbar_init(&bar_w, 1);
        mbar_init(&bar_drain, 1);
        mbar_init(&bar_stall, 1);
        mbar_init(&s_full, kWorkers);
        mbar_init(&s_free, 1);
        for (int k = 0; k < 2; ++k) {
            mbar_init(&acc_full[k], 1);
            mbar_init(&acc_empty[k], kWorkers);
        }
        abort_sh = 0;
        fence_mbar_init();
    }
    if (tid < 2) cut_sh[tid] = 0;
    if (tid == 0) flags_sh = 0;
    if (warp == kMmaWarp) tmem_alloc(&tmem_base_sh, a.tmem_cols);
    split_items(a, wsum_sh, cut_sh, cls_sm, &flags_sh, nl_sh);
    const int i0 = cut_sh[0], i1 = cut_sh[1];
    const int n_items = i1 - i0;
    const bool cls_cached = n_items <= kClsCap;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    auto cls_of = [&](int it) -> int { return cls_cached ? cls_sm[it - i0] & 3 : max(item_class(a, it), 1); };
    // First item at or after li (of this CTA) that is not lazy, n_items if none.
    auto next_nl = [&](int li) -> int {
        if (!cls_cached || li >= n_items) return min(li, n_items);
        int w = li >> 5;
        uint32_t m = nl_sh[0][w] & (0xFFFFFFFFu << (li & 31));
        const int nw = (n_items + 31) >> 5;
        while (m == 0u && ++w < nw) m = nl_sh[0][w];
        return m ? (w << 5) + __ffs(m) - 1 : n_items;
    };
    // Idle ticks deferred by item it before this tick (0 in the first tick after a reset).
    auto deferred_of = [&](int it) -> int {
        if (a.v0 || (cls_cached && !(cls_sm[it - i0] & 4))) return 0;
        return a.pend_in[it];
    };

    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (abort_sh) return false;
        if (mbar_wait_bounded(bar, parity)) return true;
        abort_sh = 1;
        atomicExch(a.err, kErrTimeout);
        return false;
    };

    if (warp < kWorkers) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kRegWorker) : "memory");
        // ------------------------------------------------------------ workers
        // Each iteration, over the CTA's items that are not lazy: (1) build
        // the operand tile S of item lc (the tensor core is idle, waiting for
        // it); (2) epilogue of the previous such item lp while the tensor core
        // works on item lc.
        //
        // Epilogue units: (neuron half h, 32-sample chunk cc).  Warp (q, g)
        // owns TMEM lanes 32q..32q+31 and units of one neuron
        // n = h*128 + 32q + lane: with two halves, h = g/2 and chunks
        // 2(g%2), 2(g%2)+1; with one half, chunk g.
        const int q = warp & 3, g = warp >> 2;
        const int nu = NH == 2 ? 2 : 1;
        const int h = NH == 2 ? (g >> 1) : 0;
        const int cc0 = NH == 2 ? (g & 1) * 2 : g;
        const int n = h * 128 + q * 32 + lane;
        constexpr int kVecs = 32 * (int)sizeof(VT) / 16;  // 16-byte vectors per 32 potentials
        constexpr bool kHalf = std::is_same<VT, __half>::value;
        // Units whose potentials are loaded before the build: one (a second
        // early unit would spill registers in every storage format).
        constexpr int kPre = 1;
        VT *Vg = reinterpret_cast<VT *>(a.V);
        // Build task of this lane: axon rax, samples 64*rhf .. 64*rhf+63 (two
        // scheduler words, read as one 8-byte vector: a warp reads 256
        // contiguous bytes of the row).
        const int tau = warp * 32 + lane;
        const bool has_task = tau < 2 * A;
        const int rax = tau >> 1, rhf = tau & 1;
        int pc = -1, bc = -1;
        int lam = 0, pth = 0, nth = 0, rst = 0;
        uint2 dd = make_uint2(0u, 0u);
        uint32_t odr = 0u;
        __half2 lam2 = __float2half2_rn(0.f), pth2 = lam2, nth2 = lam2;  // fp16 potentials only
        uint32_t rst2 = 0u;
        // Input lines of tick t that drive this lane's axon (Alg. 1: the
        // packets of the current tick are written into the scheduler before
        // the neuron block): ORed into the row words as they are read.  The
        // fan-in list [f0, f1) of the axon is kept for the current core.
        const bool has_in = a.tick < (long long)a.in_ticks;
        int fc = -1, f0 = 0, f1 = 0, ln0 = 0;
        uint2 xnext = make_uint2(0u, 0u);  // first input line's words of the next item (ORed at its build)
        auto load_words = [&](int it) -> uint2 {
            const int c = it / T, j = it % T;
            xnext = make_uint2(0u, 0u);
            if (!has_task) return make_uint2(0u, 0u);
            const uint2 *row = reinterpret_cast<const uint2 *>(a.ring + (((size_t)j * C + c) * kRows + r0) * A);
            uint2 w = row[rax * 2 + rhf];
            if (has_in) {
                if (c != fc) {
                    fc = c;
                    f0 = a.fin_ptr[(size_t)c * (A + 1) + rax];
                    f1 = a.fin_ptr[(size_t)c * (A + 1) + rax + 1];
                    ln0 = f1 > f0 ? a.fin_line[f0] : 0;
                }
                if (f1 > f0) {
                    const uint2 *in = reinterpret_cast<const uint2 *>(a.inT + ((size_t)j * a.in_ticks + a.tick) * a.Lpad) + rhf;
                    if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputLine, ln0, a.Lpad)) xnext = in[(size_t)ln0 * 2];
                    for (int e = f0 + 1; e < f1; ++e) {  // further lines (each waits for its load)
                        const int ln = a.fin_line[e];
                        if (!RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputLine, ln, a.Lpad)) continue;
                        const uint2 y = in[(size_t)ln * 2];
                        w.x |= y.x;
                        w.y |= y.y;
                    }
                }
            }
            return w;
        };
        // Class of item li of this CTA (0 past the end).
        auto cls_at = [&](int li) -> int { return li >= 0 && li < n_items ? cls_of(i0 + li) : 0; };
        // Items that are updated in this tick after deferring idle ticks: the
        // deferred ticks are applied first, each thread to the potentials that
        // its own epilogue reads later (program order, no barrier needed).
        // fn(li) for every set bit li of bitmap b (the items of this CTA).
        auto for_bits = [&](const uint32_t *b, auto &&fn) {
            for (int w = 0; w < (n_items + 31) >> 5; ++w)
                for (uint32_t m = b[w]; m; m &= m - 1u) fn((w << 5) + __ffs(m) - 1);
        };
        auto wake = [&](int li) {
            const int it = i0 + li, pe = cls_at(li) != 0 ? deferred_of(it) : 0;
            if (pe) {
                const int c = it / T, j = it % T;
                const int4 pr = a.prm[(size_t)c * N + n];
                for (int k = 0; k < nu; ++k) {
                    uint4 *vp = reinterpret_cast<uint4 *>(Vg + v_index<VT>(j, c, cc0 + k, n & ~31, 0, C, N)) + lane;
                    uint4 q[kVecs];
#pragma unroll
                    for (int e = 0; e < kVecs; ++e) q[e] = vp[e * 32];
                    defer_apply<VT>(q, (long long)pe * pr.x, pr.z);
#pragma unroll
                    for (int e = 0; e < kVecs; ++e) vp[e * 32] = q[e];
                }
            }
        };
        if (flags_sh & 1) {
            if (cls_cached) for_bits(nl_sh[1], wake);
            else for (int li = 0; li < n_items; ++li) wake(li);
        }
        // Lazy items take neither a build nor an epilogue (their tick is
        // recorded by the split); an idle item's operand is zero (its row and
        // inputs are known to be empty).  The row words of the next active
        // item are loaded right after each build, one build ahead.
        int lc = next_nl(0), lp = -1;  // item built in this iteration, item whose epilogue runs in it
        uint2 wnext = lc < n_items && cls_at(lc) == 2 ? load_words(i0 + lc) : make_uint2(0u, 0u);
        int nb = 0;  // items whose operand this warp has built (operand and accumulator phases)
        while (lc < n_items || lp >= 0) {
            // Potentials of the epilogue item lp, loaded before the build.
            const int le = lp, ite = i0 + le;
            const int ce = ite / T, je = ite % T;
            uint4 vb[kPre][kVecs];
            auto vaddr = [&](int k) {  // this lane's first 16-byte vector of unit k
                return reinterpret_cast<uint4 *>(Vg + v_index<VT>(je, ce, cc0 + k, n & ~31, 0, C, N)) + lane;
            };
            if (le >= 0) {
                if (a.v0) {  // first tick after a reset: V = v0, nothing to read
                    const uint4 vz = v_splat<VT>(a.v0[(size_t)ce * N + n]);
#pragma unroll
                    for (int k = 0; k < kPre; ++k)
#pragma unroll
                        for (int e = 0; e < kVecs; ++e) vb[k][e] = vz;
                } else {
#pragma unroll
                    for (int k = 0; k < kPre; ++k)
                        if (k < nu) {
                            const uint4 *vp = vaddr(k);
#pragma unroll
                            for (int e = 0; e < kVecs; ++e) vb[k][e] = vp[e * 32];
                        }
                }
            }
            // ---- (1) build S of item lc
            if (lc < n_items) {
                const int it = i0 + lc, c = it / T, j = it % T;
                const bool act = cls_at(lc) == 2;
                if (!wait(&s_free, (nb & 1) ^ 1)) break;
                if (c != bc) {
                    if (has_task) odr = a.outdeg[(size_t)c * A + rax];
                    bc = c;
                }
                const uint2 wrow = wnext, wcur = make_uint2(wnext.x | xnext.x, wnext.y | xnext.y);
                // Synaptic events of the item: spikes x out-degree, at most 32 * 64 * 256 per warp.
                uint32_t ev = 0u;
                if (has_task) {
                    uint2 *row = reinterpret_cast<uint2 *>(a.ring + (((size_t)j * C + c) * kRows + r0) * A);
                    if (act && (wrow.x | wrow.y)) row[rax * 2 + rhf] = make_uint2(0u, 0u);
                    const int m0 = j * 128 + rhf * 64;
                    ev = odr * (uint32_t)(__popc(wcur.x & valid_mask(a.n_valid, m0)) + __popc(wcur.y & valid_mask(a.n_valid, m0 + 32)));
                    // Row rax of the 64-sample half rhf: 8 chunks of 8 samples
                    // (16 bytes), chunk position XOR the row within its 8-axon
                    // group (128-byte swizzle).  The two halves write their
                    // chunks in opposite order, so the 8 lanes of one store
                    // phase hit 8 distinct bank groups.
                    const int r8 = rax & 7;
                    uint8_t *blk = Ssm + (size_t)(rax >> 6) * kBlockBytes + ((rax & 63) >> 3) * 2048 + rhf * 1024 + r8 * 128;
#pragma unroll
                    for (int s8 = 0; s8 < 8; ++s8) {
                        const int chunk = s8 ^ (rhf * 4);
                        const uint32_t by = (chunk < 4 ? wcur.x : wcur.y) >> (8 * (chunk & 3));
                        const uint2 lo = lut[by & 0xFu], hi = lut[(by >> 4) & 0xFu];
                        *reinterpret_cast<uint4 *>(blk + ((chunk ^ r8) << 4)) = make_uint4(lo.x, lo.y, hi.x, hi.y);
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_full);
                ++nb;
                {
                    const int ln = next_nl(lc + 1);
                    if (ln < n_items && cls_at(ln) == 2) wnext = load_words(i0 + ln);
                    else wnext = xnext = make_uint2(0u, 0u);
                }
                ev = __reduce_add_sync(0xffffffffu, ev);
                if (lane == 0 && ev) atomicAdd(a.cnt + ((size_t)j * C + c) * 4 + 3, (unsigned long long)ev);
            }
            // ---- (2) epilogue of item lp
            if (le >= 0) {
                // Items with an MMA before this one: nb counts those up to item lc.
                const int ne = nb - (lc < n_items ? 1 : 0) - 1;
                const int buf = ne & 1;
                if (ce != pc) {
                    const int4 pr = a.prm[(size_t)ce * N + n];  // leak, pos_thr, neg_thr, reset
                    // folds the bias of f32_bits_minus_bias; wrap-around (unsigned)
                    // arithmetic: the sum below is exact whenever V + dV + leak fits int32
                    lam = (int)((uint32_t)pr.x - 0x4B400000u);
                    pth = pr.y;
                    nth = pr.z;
                    rst = pr.w;
                    if constexpr (kHalf) {  // every one of these is an integer of magnitude <= 2048: exact
                        lam2 = __float2half2_rn((float)pr.x);
                        pth2 = __float2half2_rn((float)pr.y);
                        nth2 = __float2half2_rn((float)pr.z);
                        const __half2 r2 = __float2half2_rn((float)pr.w);
                        rst2 = *reinterpret_cast<const uint32_t *>(&r2);
                    }
                    dd = a.dst[(size_t)ce * N + n];
                    pc = ce;
                }
                if (!wait(&acc_full[buf], (ne >> 1) & 1)) break;
                tc_fence_after();
                const uint32_t kind = dest_kind(dd);
                uint32_t n_sp = 0, n_pk = 0, n_out = 0;
                uint32_t dm0 = 0u, dm1 = 0u;  // spike masks of the two units (delivered together when nu == 2)
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (k >= nu) break;
                    const int cc = cc0 + k;
                    if (k >= kPre) {
                        if (a.v0) {
                            const uint4 vz = v_splat<VT>(a.v0[(size_t)ce * N + n]);
#pragma unroll
                            for (int e = 0; e < kVecs; ++e) vb[k % kPre][e] = vz;
                        }  // otherwise loaded during the first unit, half by half
                    }
                    uint4 *vout = vaddr(k);
                    uint32_t mask = 0u;
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        __syncwarp();
                        uint32_t d[16];
                        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * NH * 128 + h * 128 + cc * 32 + hf * 16), d);
                        if constexpr (kHalf) {
                            // Pairs of samples.  V + leak is exact in fp16, the
                            // sum with dV exact in fp32; rounding that sum to
                            // fp16 is monotone and keeps every integer of
                            // magnitude <= 2048, so with both thresholds and
                            // their predecessors representable the comparisons
                            // decide as on the integers, and a value that is kept
                            // (theta- <= x < theta+) is exact.  Overflow to
                            // +-inf compares the same way.
                            uint32_t wv[8];
#pragma unroll
                            for (int q2 = 0; q2 < 2; ++q2) {
                                const uint4 u = vb[k % kPre][hf * 2 + q2];
                                wv[4 * q2] = u.x;
                                wv[4 * q2 + 1] = u.y;
                                wv[4 * q2 + 2] = u.z;
                                wv[4 * q2 + 3] = u.w;
                            }
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const float2 vl = __half22float2(__hadd2(*reinterpret_cast<const __half2 *>(&wv[e]), lam2));
                                const __half2 x2 = __floats2half2_rn(__uint_as_float(d[2 * e]) + vl.x,
                                                                     __uint_as_float(d[2 * e + 1]) + vl.y);
                                const uint32_t fm = __hge2_mask(x2, pth2);
                                uint32_t keep;
                                if constexpr (kNegReset) {
                                    const uint32_t rm = fm | __hlt2_mask(x2, nth2);
                                    keep = *reinterpret_cast<const uint32_t *>(&x2);
                                    wv[e] = (rm & rst2) | (~rm & keep);
                                } else {
                                    const __half2 c2 = __hmax2(x2, nth2);
                                    keep = *reinterpret_cast<const uint32_t *>(&c2);
                                    wv[e] = (fm & rst2) | (~fm & keep);
                                }
                                mask |= ((fm & 1u) | ((fm >> 15) & 2u)) << (hf * 16 + 2 * e);
                            }
                            vout[(hf * 2) * 32] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                            vout[(hf * 2 + 1) * 32] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
                        } else {
                            int v[16];
                            unpack16<VT>(vb[k % kPre], hf, v);
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const int x = (int)((uint32_t)v[i] + (uint32_t)f32_bits_minus_bias(d[i]) + (uint32_t)lam);
                                const bool fire = x >= pth;
                                int y = kNegReset ? (x < nth ? rst : x) : max(x, nth);
                                y = fire ? rst : y;
                                v[i] = y;
                                mask |= (fire ? 1u : 0u) << (hf * 16 + i);
                            }
                            store16<VT>(vout, hf, v);
                        }
                        if (k == 0 && nu == 2 && !a.v0) {  // this half's vectors are free: the second unit's
                            const uint4 *vp1 = vaddr(1);
#pragma unroll
                            for (int e = 0; e < kVecs / 2; ++e) vb[0][hf * (kVecs / 2) + e] = vp1[(hf * (kVecs / 2) + e) * 32];
                        }
                    }
                    a.spk[(((size_t)je * C + ce) * 4 + cc) * N + n] = mask;
                    const uint32_t valid = valid_mask(a.n_valid, je * 128 + cc * 32);
                    const uint32_t live = mask & valid;
                    n_sp += __popc(live);
                    if (mask && kind == RANC_DEST_CORE) {
                        n_pk += __popc(live);
                        if (nu == 1 && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestCore, dd.x, C) &&
                            RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestAxon, dest_axon(dd), A)) {
                            const uint32_t ax = dest_axon(dd);
                            const int r = (int)((a.tick + dest_delay(dd)) & (kRows - 1));
                            atomicOr(reinterpret_cast<uint32_t *>(a.ring) + ((((size_t)je * C + dd.x) * kRows + r) * A + ax) * 4 + cc,
                                     mask);
                            // The destination row's stamp: the cycle of the tick that reads it.
                            a.stamp[(size_t)r * a.spitch + (size_t)dd.x * T + je] = (uint8_t)((a.sclock + dest_delay(dd)) >> 4);
                        }
                    }
                    (k == 0 ? dm0 : dm1) = mask;
                    // Output bus: one warp-wide pass per output neuron that fired;
                    // lane i adds sample cc*32 + i, so no lane loops over spikes.
                    uint32_t olanes = __ballot_sync(0xffffffffu, kind == RANC_DEST_OUTPUT && live != 0u);
                    if (kind == RANC_DEST_OUTPUT) n_out += __popc(live);
                    while (olanes) {
                        const int L = __ffs(olanes) - 1;
                        olanes &= olanes - 1u;
                        const uint32_t mL = __shfl_sync(0xffffffffu, live, L);
                        const uint32_t idL = __shfl_sync(0xffffffffu, dd.x, L);
                        const int bs = je * 128 + cc * 32 + lane;
                        if (((mL >> lane) & 1u) && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteOutputId, idL, a.n_out)) {
                            atomicAdd(a.out + (size_t)bs * a.n_out + idL, 1u);
                            if (a.olog && bs < a.olog_rows) atomicAdd(a.olog + (size_t)bs * a.olog_stride + idL, 1u);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[buf]);
                // Two units of one neuron: adjacent words (cc0 even) of the same
                // destination row, delivered by one 64-bit atomicOr, one stamp.
                if (nu == 2 && kind == RANC_DEST_CORE && (dm0 | dm1) && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestCore, dd.x, C) &&
                    RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestAxon, dest_axon(dd), A)) {
                    const uint32_t ax = dest_axon(dd);
                    const int r = (int)((a.tick + dest_delay(dd)) & (kRows - 1));
                    atomicOr(reinterpret_cast<unsigned long long *>(reinterpret_cast<uint32_t *>(a.ring) +
                                                                    ((((size_t)je * C + dd.x) * kRows + r) * A + ax) * 4 + cc0),
                             ((unsigned long long)dm1 << 32) | dm0);
                    a.stamp[(size_t)r * a.spitch + (size_t)dd.x * T + je] = (uint8_t)((a.sclock + dest_delay(dd)) >> 4);
                }
                n_sp = __reduce_add_sync(0xffffffffu, n_sp);
                n_pk = __reduce_add_sync(0xffffffffu, n_pk);
                n_out = __reduce_add_sync(0xffffffffu, n_out);
                if (lane == 0 && (n_sp | n_pk | n_out)) {
                    unsigned long long *cp = a.cnt + ((size_t)je * C + ce) * 4;
                    atomicAdd(cp + 0, (unsigned long long)n_sp);
                    atomicAdd(cp + 1, (unsigned long long)n_pk);
                    atomicAdd(cp + 2, (unsigned long long)n_out);
                }
            }
            lp = lc < n_items ? lc : -1;
            lc = next_nl(lc + 1);
        }
    } else {
      asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kRegIssuer) : "memory");
      if (warp == kMmaWarp && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        int loaded = -1;
        uint32_t nw = 0, nd = 0;
        bool w_pending = false;
        const size_t vtile = (size_t)4 * N * 32 * sizeof(VT);
        int na = 0;  // items issued, in the order the workers build them
        int lc = next_nl(0);
        int l1 = lc < n_items ? next_nl(lc + 1) : n_items;
        for (; lc < n_items; lc = l1, l1 = l1 < n_items ? next_nl(l1 + 1) : n_items) {
            const int it = i0 + lc, c = it / T, buf = na & 1;
            const bool act = cls_of(it) == 2;
            if (c != loaded) {
                if (loaded >= 0) {  // every MMA reading the old weights has finished
                    mma_commit(&bar_drain);
                    if (!wait(&bar_drain, nd & 1)) break;
                    ++nd;
                }
                mbar_arrive_expect_tx(&bar_w, (uint32_t)N * A * 2);
                for (int hh = 0; hh < NH; ++hh)
                    for (int kb = 0; kb < KB; ++kb)
                        tma_load_3d(Wsm + (size_t)(hh * KB + kb) * kBlockBytes, &wmap, kb * 64, hh * 128, c, &bar_w);
                w_pending = true;
                uint64_t *wbar = &bar_w;
                uint32_t wpar = nw & 1;
                if (a.stall_test && blockIdx.x == 0 && nw == 0) {
                    // Failure-detection test: the wait is moved to a barrier that
                    // expects 16 bytes no copy delivers; it runs out, and the
                    // weight copies just issued land (drain below) before exit.
                    mbar_arrive_expect_tx(&bar_stall, 16u);
                    wbar = &bar_stall;
                    wpar = 0;
                }
                if (!wait(wbar, wpar)) break;
                w_pending = false;
                ++nw;
                loaded = c;
            }
            if (l1 < n_items) {  // potentials of the next item
                const int c1 = (i0 + l1) / T, j1 = (i0 + l1) % T;
                prefetch_l2(reinterpret_cast<const uint8_t *>(a.V) + ((size_t)j1 * C + c1) * vtile, (uint32_t)vtile);
                const int l2 = next_nl(l1 + 1);
                if (l2 < n_items && cls_of(i0 + l2) == 2) {  // scheduler row of the one after
                    const int c2 = (i0 + l2) / T, j2 = (i0 + l2) % T;
                    prefetch_l2(a.ring + (((size_t)j2 * C + c2) * kRows + r0) * A, (uint32_t)A * 16u);
                }
            }
            if (!wait(&acc_empty[buf], ((na >> 1) & 1) ^ 1)) break;
            if (!wait(&s_full, na & 1)) break;
            tc_fence_after();
            if (!act) {  // idle: the zero operand's first K-step gives dV = 0
                for (int hh = 0; hh < NH; ++hh)
                    mma_f16(tmem + (uint32_t)(buf * NH * 128 + hh * 128), smem_desc_kmajor(smem_u32(Wsm + (size_t)hh * KB * kBlockBytes)),
                            smem_desc_mn(smem_u32(Ssm)), false);
            } else
            for (int kb = 0; kb < KB; ++kb) {
#pragma unroll 1
                for (int hh = 0; hh < NH; ++hh) {
                    const uint32_t d = tmem + (uint32_t)(buf * NH * 128 + hh * 128);
                    const uint32_t wa = smem_u32(Wsm + (size_t)(hh * KB + kb) * kBlockBytes);
                    const uint32_t sb = smem_u32(Ssm + (size_t)kb * kBlockBytes);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)  // K = 16: 32 bytes along a weight row, two 8-axon groups of S
                        mma_f16(d, smem_desc_kmajor(wa + ks * 32), smem_desc_mn(sb + ks * 4096), (kb | ks) != 0);
                }
            }
            mma_commit(&s_free);
            mma_commit(&acc_full[buf]);
            ++na;
        }
        // Drain: all MMAs issued by this thread complete before tensor memory is freed.
        mma_commit(&bar_drain);
        mbar_wait_bounded(&bar_drain, nd & 1);
        if (w_pending) mbar_wait_bounded(&bar_w, nw & 1);  // a weight load still in flight
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) tmem_dealloc(tmem, a.tmem_cols);
}

// ---------------------------------------------------------------------------
// Helper kernels: reset, input transposition, state export / import
// ---------------------------------------------------------------------------

// V <- v0: every 16-byte vector holds samples of one (tile, core, neuron), so
// it is v0 of that neuron repeated.  Vector e of the interleaved layout:
// e = (((j*C + c)*4 + cc)*(N/32) + n/32)*P + p)*32 + n%32.
template <typename VT>
__global__ void batched_reset_v(VT *V, const int *v0, int C, int N, long long vecs) {
    constexpr int P = 32 * (int)sizeof(VT) / 16;
    uint4 *p = reinterpret_cast<uint4 *>(V);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < vecs; e += (long long)gridDim.x * blockDim.x) {
        const long long g = e / (32 * P);  // ((j*C + c)*4 + cc)*(N/32) + n/32
        const int n = (int)(g % (N / 32)) * 32 + (int)(e % 32);
        const int c = (int)((g / (N / 32) / 4) % C);
        const VT x = v_from_int<VT>(v0[(size_t)c * N + n]);
        uint32_t w;
        if constexpr (sizeof(VT) == 2) w = (uint32_t)(*reinterpret_cast<const uint16_t *>(&x)) * 0x10001u;
        else w = (uint32_t)x;
        p[e] = make_uint4(w, w, w, w);
    }
}

// Applies the idle ticks that lazy items deferred: V <- max(V + k * leak,
// theta-) for k = pend[c * T + j] (exact: the result lies in [theta-, V];
// formed in 64 bits, since k * leak may not fit 32), and clears their spike
// masks (a lazy tick fires nothing; the tick kernel leaves them as they were).
// Vector e of the interleaved layout as in batched_reset_v; spike word w of
// spk [T][C][4][N].
template <typename VT>
__global__ void batched_catch_up(VT *V, uint32_t *spk, const uint8_t *pend, const int4 *prm, int C, int N, int T, long long vecs) {
    const long long words = (long long)T * C * 4 * N;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < words; w += (long long)gridDim.x * blockDim.x) {
        const long long jc = w / (4 * N);
        const int c = (int)(jc % C), j = (int)(jc / C);
        if (pend[(size_t)c * T + j]) spk[w] = 0u;
    }
    constexpr int P = 32 * (int)sizeof(VT) / 16, E = 16 / (int)sizeof(VT);
    uint4 *p = reinterpret_cast<uint4 *>(V);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < vecs; e += (long long)gridDim.x * blockDim.x) {
        const long long g = e / (32 * P);  // ((j*C + c)*4 + cc)*(N/32) + n/32
        const int n = (int)(g % (N / 32)) * 32 + (int)(e % 32);
        const long long jc = g / (N / 32) / 4;
        const int c = (int)(jc % C), j = (int)(jc / C);
        const int k = pend[(size_t)c * T + j];
        if (k == 0) continue;
        const int4 pr = prm[(size_t)c * N + n];
        uint4 u = p[e];
        VT *x = reinterpret_cast<VT *>(&u);
#pragma unroll
        for (int i = 0; i < E; ++i) x[i] = v_from_int<VT>((int)max((long long)v_to_int<VT>(x[i]) + (long long)k * pr.x, (long long)pr.z));
        p[e] = u;
    }
}

// x [n_samples][ticks][words] -> inT [T][ticks][Lpad][4] (sample-minor).
__global__ void transpose_inputs(const uint32_t *x, int n_samples, int ticks, int words, int T, uint32_t *inT) {
    const int lane = threadIdx.x & 31;
    const long long task = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long n_tasks = (long long)T * ticks * words * 4;
    if (task >= n_tasks) return;
    const int w = (int)(task % 4);
    const int lb = (int)((task / 4) % words);
    const int t = (int)((task / 4 / words) % ticks);
    const int j = (int)(task / 4 / words / ticks);
    const int s = j * 128 + w * 32 + lane;
    const uint32_t word = s < n_samples ? x[((size_t)s * ticks + t) * words + lb] : 0u;
    const uint32_t y = transpose32(word, lane);
    inT[((((size_t)j * ticks + t) * words * 32) + lb * 32 + lane) * 4 + w] = y;
}

// Canonical copies of samples [b0, b0 + nb): v [nb][C][N], spk [nb][C][N/32],
// ring [nb][C][16][A/32] (ring may be NULL).
template <typename VT>
__global__ void export_state(const VT *Vb, const uint32_t *spkb, const uint32_t *ringb, int b0, int nb, int C, int N,
                             int A, int *v, uint32_t *spk, uint32_t *ring) {
    const long long nv = (long long)nb * C * N, ns = (long long)nb * C * (N / 32),
                    nr = ring ? (long long)nb * C * kRows * (A / 32) : 0;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nv + ns + nr;
         f += (long long)gridDim.x * blockDim.x) {
        if (f < nv) {
            const int n = (int)(f % N), c = (int)((f / N) % C), b = b0 + (int)(f / N / C);
            const int j = b >> 7, cc = (b & 127) >> 5, i = b & 31;
            v[f] = v_to_int<VT>(Vb[v_index<VT>(j, c, cc, n, i, C, N)]);
        } else if (f < nv + ns) {
            const long long g = f - nv;
            const int wn = (int)(g % (N / 32)), c = (int)((g / (N / 32)) % C), b = b0 + (int)(g / (N / 32) / C);
            const int j = b >> 7, cc = (b & 127) >> 5, i = b & 31;
            uint32_t word = 0;
            for (int k = 0; k < 32; ++k)
                word |= ((spkb[(((size_t)j * C + c) * 4 + cc) * N + wn * 32 + k] >> i) & 1u) << k;
            spk[g] = word;
        } else {
            const long long g = f - nv - ns;
            const int AW = A / 32;
            const int aw = (int)(g % AW), r = (int)((g / AW) % kRows), c = (int)((g / AW / kRows) % C),
                      b = b0 + (int)(g / AW / kRows / C);
            const int j = b >> 7, cc = (b & 127) >> 5, i = b & 31;
            uint32_t word = 0;
            for (int k = 0; k < 32; ++k)
                word |= ((ringb[((((size_t)j * C + c) * kRows + r) * A + aw * 32 + k) * 4 + cc] >> i) & 1u) << k;
            ring[g] = word;
        }
    }
}

template <typename VT>
__global__ void import_state(VT *Vb, uint32_t *spkb, uint32_t *ringb, int B, int T, int C, int N, int A, const int *v,
                             const uint32_t *spk, const uint32_t *ring) {
    const long long nv = (long long)B * C * N, ns = (long long)T * C * 4 * N, nr = (long long)T * C * kRows * A * 4;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nv + ns + nr;
         f += (long long)gridDim.x * blockDim.x) {
        if (f < nv) {
            const int n = (int)(f % N), c = (int)((f / N) % C), b = (int)(f / N / C);
            const int j = b >> 7, cc = (b & 127) >> 5, i = b & 31;
            Vb[v_index<VT>(j, c, cc, n, i, C, N)] = v_from_int<VT>(v[f]);
        } else if (f < nv + ns) {
            const long long g = f - nv;  // ((j*C + c)*4 + cc)*N + n
            const int n = (int)(g % N), cc = (int)((g / N) % 4), c = (int)((g / N / 4) % C), j = (int)(g / N / 4 / C);
            uint32_t word = 0;
            for (int i = 0; i < 32; ++i) {
                const int b = j * 128 + cc * 32 + i;
                if (b < B) word |= ((spk[((size_t)b * C + c) * (N / 32) + n / 32] >> (n & 31)) & 1u) << i;
            }
            spkb[g] = word;
        } else {
            const long long g = f - nv - ns;  // (((j*C + c)*16 + r)*A + a)*4 + cc
            const int cc = (int)(g % 4), ax = (int)((g / 4) % A), r = (int)((g / 4 / A) % kRows),
                      c = (int)((g / 4 / A / kRows) % C), j = (int)(g / 4 / A / kRows / C);
            uint32_t word = 0;
            for (int i = 0; i < 32; ++i) {
                const int b = j * 128 + cc * 32 + i;
                if (b < B)
                    word |= ((ring[(((size_t)b * C + c) * kRows + r) * (A / 32) + ax / 32] >> (ax & 31)) & 1u) << i;
            }
            ringb[g] = word;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct Batched {
    int NH = 0, KB = 0, Lpad = 0, n_sm = 0;
    uint32_t tmem_cols = 0;
    size_t smem = 0;
    __half *wfold = nullptr;
    int *fin_ptr = nullptr, *fin_line = nullptr;
    uint32_t *outdeg = nullptr;
    uint4 *inT = nullptr;
    size_t inT_cap = 0;
    // Item activity: delivery stamps [16][spitch], deferred idle ticks
    // [2][spitch] (double-buffered by tick parity), per-core flags.
    uint8_t *stamp = nullptr, *pend = nullptr, *core_flags = nullptr;
    unsigned long long *item_ticks = nullptr;  // [3] updated / deferred / active item-ticks since the last counter reset
    long long spitch = 0;
    bool any_lazy = false;
    // Relative cost of an active, idle and lazy item, of applying deferred
    // ticks and of the output-bus events of an updated item of an output
    // core; the split of a tick's items over the CTAs balances their sum.
    // Per-CTA busy times of the 512-core MNIST-shaped window against the
    // CTAs' item mix give about 4.3 us per active item, 3.5 us per idle one,
    // 18 ns per lazy one, 2.9 us to apply deferred ticks, and 0-1 us more per
    // item of an output core (growing with its output-bus events).
    int cost_active = 256, cost_idle = 208, cost_lazy = 1, cost_wake = 168, cost_out = 32;
    CUtensorMap wmap;  // 64-byte aligned by its declaration
};

Batched *B_of(ranc_sim *s) { return static_cast<Batched *>(s->tmap); }

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

long long grid_for(long long n) { return std::max<long long>(1, std::min<long long>((n + 255) / 256, 8192)); }

}  // namespace

// Storage of the potentials on the batched paths.  After a tick a neuron
// holds v0 (before its first tick), its reset value, theta-, or a value x
// with theta- <= x < theta+, so every stored value lies in [lo, hi] below.
// int16 holds that range exactly when it fits.  fp16 is exact for the update
// (the tick kernels' fp16 branch) when [lo, hi] and [lo, hi] + leak lie
// within +-2048 (every integer there is an fp16 value) and theta+, theta+ - 1,
// theta-, theta- - 1 and the leak are representable.
int potential_format_of(const ranc_desc *d) {
    bool fits16 = true, fitsh = true;
    for (size_t i = 0; i < (size_t)d->n_cores * d->neurons; i++) {
        const long long pt = d->pos_thr[i], nt = d->neg_thr[i], r = d->reset[i], v0 = d->v0[i], lk = d->leak[i];
        const long long hi = std::max({pt - 1, nt, r, v0});
        const long long lo = std::min({nt, r, v0});
        if (hi > 32767 || lo < -32768) fits16 = false;
        if (lo < -2048 || hi > 2048 || lo + lk < -2048 || hi + lk > 2048 || lk < -2048 || lk > 2048 || pt < -2047 ||
            pt > 2048 || nt < -2047 || nt > 2048)
            fitsh = false;
    }
    return fitsh ? kVHalf : fits16 ? kVInt16 : kVInt32;
}

cudaError_t batched_setup(ranc_sim *sim, const ranc_desc *d, std::string &why) {
    const int C = d->n_cores, A = d->axons, N = d->neurons, K = d->n_types;
    if (!(N == 128 || N == 256) || A % 64 != 0 || A < 64 || A > 256) {
        why = "the batched path needs neurons in {128, 256} and axons a multiple of 64 in [64, 256]";
        return cudaErrorInvalidValue;
    }
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, sim->device);
    if (e != cudaSuccess) {
        why = "cudaGetDeviceProperties";
        return e;
    }
    if (prop.major != 10 || prop.minor != 3) {
        why = "the batched path needs an sm_103 (GB300) device";
        return cudaErrorInvalidValue;
    }
    Batched *bs = new (std::nothrow) Batched();
    if (!bs) {
        why = "host allocation";
        return cudaErrorMemoryAllocation;
    }
    sim->tmap = bs;
    bs->NH = N / 128;
    bs->KB = A / 64;
    bs->Lpad = sim->in_words * 32;
    bs->n_sm = prop.multiProcessorCount;
    bs->tmem_cols = bs->NH == 2 ? 512u : 256u;
    bs->smem = (size_t)(bs->NH + 1) * bs->KB * kBlockBytes + 256 * 16 + kClsCap + 1024;
    sim->T = (sim->B + kTileS - 1) / kTileS;
    sim->B_pad = sim->T * kTileS;

    sim->vmode = potential_format_of(d);
    // Largest delay of a core-to-core packet: bounds the scheduler rows that
    // can still hold deliveries when the handle is reset.
    sim->max_delay = 0;
    for (size_t i = 0; i < (size_t)C * N; i++)
        if (d->dest[i].kind == RANC_DEST_CORE) sim->max_delay = std::max<int>(sim->max_delay, d->dest[i].delay);

    // Folded weights W[c][n][a] = connected(a, n) ? w[type(a)][n] : 0 (fp16, exact).
    std::vector<__half> wf((size_t)C * N * A);
    std::vector<uint32_t> od((size_t)C * A, 0);
    const int NWd = N / 32;
    for (int c = 0; c < C; c++)
        for (int ax = 0; ax < A; ax++) {
            const uint32_t *row = d->crossbar + ((size_t)c * A + ax) * NWd;
            const int k = d->axon_type[(size_t)c * A + ax];
            for (int n = 0; n < N; n++) {
                const bool on = (row[n >> 5] >> (n & 31)) & 1u;
                wf[((size_t)c * N + n) * A + ax] = __float2half((float)(on ? d->weight[((size_t)c * K + k) * N + n] : 0));
                od[(size_t)c * A + ax] += on ? 1 : 0;
            }
        }
    // Input fan-in per (core, axon).
    std::vector<int> fptr((size_t)C * (A + 1), 0), fline;
    {
        std::vector<std::vector<int>> lists((size_t)C * A);
        const int nnz = d->n_inputs > 0 ? d->in_offsets[d->n_inputs] : 0;
        (void)nnz;
        for (int i = 0; i < d->n_inputs; i++)
            for (int k = d->in_offsets[i]; k < d->in_offsets[i + 1]; k++)
                lists[(size_t)d->in_core[k] * A + d->in_axon[k]].push_back(i);
        for (int c = 0; c < C; c++) {
            for (int ax = 0; ax < A; ax++) {
                fptr[(size_t)c * (A + 1) + ax] = (int)fline.size();
                for (int L : lists[(size_t)c * A + ax]) fline.push_back(L);
            }
            fptr[(size_t)c * (A + 1) + A] = (int)fline.size();
        }
        if (fline.empty()) fline.push_back(0);
    }
    // Per core: driven by an input line; idle ticks deferrable (item_class);
    // drives the output bus (split cost).
    std::vector<uint8_t> cfl(C, 0);
    for (int c = 0; c < C; c++) {
        const bool driven = fptr[(size_t)c * (A + 1) + A] > fptr[(size_t)c * (A + 1)];
        bool ok = d->neg_mode == 0;
        for (int n = 0; n < N && ok; n++) {
            const size_t i = (size_t)c * N + n;
            const long long pt = d->pos_thr[i];
            ok = d->leak[i] <= 0 && d->neg_thr[i] < pt && d->reset[i] < pt && d->v0[i] < pt;
        }
        bool out = false;
        for (int n = 0; n < N && !out; n++) out = d->dest[(size_t)c * N + n].kind == RANC_DEST_OUTPUT;
        cfl[c] = (uint8_t)((driven ? 1 : 0) | (ok ? 2 : 0) | (out ? 4 : 0));
        bs->any_lazy = bs->any_lazy || ok;
    }
    bs->spitch = ((long long)sim->T * C + 127) / 128 * 128;
    const size_t vsz = sim->vmode == kVInt32 ? 4 : 2;
    if (dev_alloc((void **)&bs->wfold, wf.size() * 2) != cudaSuccess || dev_alloc((void **)&bs->outdeg, od.size() * 4) != cudaSuccess ||
        dev_alloc((void **)&bs->fin_ptr, fptr.size() * 4) != cudaSuccess ||
        dev_alloc((void **)&bs->fin_line, fline.size() * 4) != cudaSuccess ||
        dev_alloc((void **)&sim->V, (size_t)sim->T * C * 4 * N * 32 * vsz) != cudaSuccess ||
        dev_alloc((void **)&sim->ring, (size_t)sim->T * C * kRows * A * 16) != cudaSuccess ||
        dev_alloc((void **)&sim->spk, (size_t)sim->T * C * 4 * N * 4) != cudaSuccess ||
        dev_alloc((void **)&sim->out, (size_t)sim->B_pad * sim->n_outputs * 4) != cudaSuccess ||
        dev_alloc((void **)&sim->cnt, (size_t)sim->T * C * 4 * 8) != cudaSuccess ||
        dev_alloc((void **)&bs->stamp, (size_t)kRows * bs->spitch) != cudaSuccess ||
        dev_alloc((void **)&bs->pend, (size_t)2 * bs->spitch) != cudaSuccess ||
        dev_alloc((void **)&bs->core_flags, (size_t)C) != cudaSuccess || dev_alloc((void **)&bs->item_ticks, 24) != cudaSuccess) {
        why = "device allocation of the batched state failed";
        return cudaErrorMemoryAllocation;
    }
    sim->cnt_len = (size_t)sim->T * C * 4;
    if ((e = cudaMemcpy(bs->wfold, wf.data(), wf.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(bs->outdeg, od.data(), od.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(bs->fin_ptr, fptr.data(), fptr.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(bs->fin_line, fline.data(), fline.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(bs->core_flags, cfl.data(), (size_t)C, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(bs->stamp, 0, (size_t)kRows * bs->spitch)) != cudaSuccess ||
        (e = cudaMemset(bs->pend, 0, (size_t)2 * bs->spitch)) != cudaSuccess ||
        (e = cudaMemset(bs->item_ticks, 0, 24)) != cudaSuccess) {
        why = "copy of the batched network arrays";
        return e;
    }

    // Tensor map of the folded weights: dims (A, N, C), box (64, 128, 1), 128-byte swizzle.
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if ((e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q)) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        why = "cuTensorMapEncodeTiled is unavailable";
        return e != cudaSuccess ? e : cudaErrorNotSupported;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)A, (cuuint64_t)N, (cuuint64_t)C};
    const cuuint64_t strides[2] = {(cuuint64_t)A * 2, (cuuint64_t)N * A * 2};
    const cuuint32_t box[3] = {64, 128, 1}, estr[3] = {1, 1, 1};
    CUresult cr = reinterpret_cast<EncodeTiledFn>(fn)(&bs->wmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, bs->wfold, dims,
                                                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        why = "cuTensorMapEncodeTiled failed";
        return cudaErrorInvalidValue;
    }
    // The attribute belongs to the kernel, not to this handle: it is only ever
    // raised, so handles of different shapes can coexist in one process.
    const int sm = (int)bs->smem;
    if ((e = raise_smem_limit((const void *)batched_tick_kernel<__half, 0>, sm)) != cudaSuccess ||
        (e = raise_smem_limit((const void *)batched_tick_kernel<__half, 1>, sm)) != cudaSuccess ||
        (e = raise_smem_limit((const void *)batched_tick_kernel<int16_t, 0>, sm)) != cudaSuccess ||
        (e = raise_smem_limit((const void *)batched_tick_kernel<int16_t, 1>, sm)) != cudaSuccess ||
        (e = raise_smem_limit((const void *)batched_tick_kernel<int, 0>, sm)) != cudaSuccess ||
        (e = raise_smem_limit((const void *)batched_tick_kernel<int, 1>, sm)) != cudaSuccess)
        why = "kernel shared-memory attribute";
    return e;
}

cudaError_t launch_batched_tick(ranc_sim *sim, const BatchedArgs &) {
    Batched *bs = B_of(sim);
    TickArgs a{};
    a.C = sim->C; a.A = sim->A; a.N = sim->N; a.NH = bs->NH; a.KB = bs->KB; a.T = sim->T;
    a.n_valid = sim->n_valid; a.Lpad = bs->Lpad; a.in_ticks = bs->inT ? sim->in_ticks : 0; a.n_out = sim->n_outputs;
    a.neg_mode = sim->neg_mode; a.items = sim->T * sim->C; a.tick = sim->tick;
    a.prm = sim->prm; a.dst = sim->dst; a.fin_ptr = bs->fin_ptr; a.fin_line = bs->fin_line; a.outdeg = bs->outdeg;
    a.inT = bs->inT; a.v0 = sim->v_lazy ? sim->v0 : nullptr; a.V = sim->V; a.ring = reinterpret_cast<uint4 *>(sim->ring); a.spk = sim->spk; a.out = sim->out;
    a.cnt = sim->cnt; a.err = sim->err; a.tmem_cols = bs->tmem_cols;
    a.olog = sim->olog_t; a.olog_stride = sim->olog_stride; a.olog_rows = sim->B;
    // The stamp clock runs with the tick modulo 16 (a reset moves it to the
    // next multiple of 16).  If the tick was set otherwise (a state import),
    // the clock jumps ahead and every item counts as active until all rows
    // written under the old clock have been read.
    if (((sim->sclock ^ (uint32_t)sim->tick) & (kRows - 1)) != 0) {
        sim->sclock = ((sim->sclock + 2 * kRows) & ~(uint32_t)(kRows - 1)) | ((uint32_t)sim->tick & (kRows - 1));
        sim->all_active_ticks = kRows;
    }
    a.stamp = bs->stamp; a.spitch = bs->spitch; a.stamp_row = bs->stamp + (size_t)(sim->tick & (kRows - 1)) * bs->spitch;
    a.sclock = sim->sclock; a.all_active = sim->all_active_ticks > 0;
    a.core_flags = bs->core_flags;
    a.pend_in = bs->pend + (size_t)(sim->tick & 1) * bs->spitch;
    a.pend_out = bs->pend + (size_t)((sim->tick + 1) & 1) * bs->spitch;
    a.cost_active = bs->cost_active; a.cost_idle = bs->cost_idle; a.cost_lazy = bs->cost_lazy; a.cost_wake = bs->cost_wake;
    a.cost_out = bs->cost_out;
    a.item_ticks = bs->item_ticks;
    a.stall_test = sim->stall_test;
    a.dbg_plant = sim->dbg_plant;
    const int grid = std::min(bs->n_sm, a.items);
    auto kern = sim->vmode == kVHalf    ? (sim->neg_mode ? batched_tick_kernel<__half, 1> : batched_tick_kernel<__half, 0>)
                : sim->vmode == kVInt16 ? (sim->neg_mode ? batched_tick_kernel<int16_t, 1> : batched_tick_kernel<int16_t, 0>)
                                        : (sim->neg_mode ? batched_tick_kernel<int, 1> : batched_tick_kernel<int, 0>);
    kern<<<grid, kThreads, bs->smem, sim->stream>>>(a, bs->wmap);
    sim->v_lazy = 0;  // this tick wrote V and the spike masks
    sim->sclock++;
    if (sim->all_active_ticks > 0) --sim->all_active_ticks;
    if (bs->any_lazy) sim->pend_dirty = 1;
    return cudaGetLastError();
}

// V <- v0 and no spikes: materialised only when something reads the state
// before the first tick after a reset (that tick reads v0 itself).
static cudaError_t batched_materialize(ranc_sim *sim) {
    Batched *bs = B_of(sim);
    uint8_t *pend_cur = bs->pend + (size_t)(sim->tick & 1) * bs->spitch;  // what the next tick reads
    if (!sim->v_lazy) {
        if (!sim->pend_dirty) return cudaSuccess;
        const long long vecs = (long long)sim->T * sim->C * 4 * sim->N * (sim->vmode == kVInt32 ? 8 : 4);
        const unsigned g = (unsigned)grid_for(vecs);
        if (sim->vmode == kVHalf)
            batched_catch_up<__half><<<g, 256, 0, sim->stream>>>((__half *)sim->V, sim->spk, pend_cur, sim->prm, sim->C, sim->N, sim->T, vecs);
        else if (sim->vmode == kVInt16)
            batched_catch_up<int16_t><<<g, 256, 0, sim->stream>>>((int16_t *)sim->V, sim->spk, pend_cur, sim->prm, sim->C, sim->N, sim->T, vecs);
        else
            batched_catch_up<int><<<g, 256, 0, sim->stream>>>((int *)sim->V, sim->spk, pend_cur, sim->prm, sim->C, sim->N, sim->T, vecs);
        sim->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(pend_cur, 0, (size_t)bs->spitch, sim->stream)) != cudaSuccess) return e;
        sim->pend_dirty = 0;
        return cudaSuccess;
    }
    if (cudaError_t e = cudaMemsetAsync(pend_cur, 0, (size_t)bs->spitch, sim->stream); e != cudaSuccess) return e;
    sim->pend_dirty = 0;
    const long long total = (long long)sim->T * sim->C * 4 * sim->N * (sim->vmode == kVInt32 ? 8 : 4);  // 16-byte vectors
    if (sim->vmode == kVHalf)
        batched_reset_v<__half><<<(unsigned)grid_for(total), 256, 0, sim->stream>>>((__half *)sim->V, sim->v0, sim->C, sim->N, total);
    else if (sim->vmode == kVInt16)
        batched_reset_v<int16_t><<<(unsigned)grid_for(total), 256, 0, sim->stream>>>((int16_t *)sim->V, sim->v0, sim->C, sim->N, total);
    else
        batched_reset_v<int><<<(unsigned)grid_for(total), 256, 0, sim->stream>>>((int *)sim->V, sim->v0, sim->C, sim->N, total);
    sim->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sim->spk, 0, (size_t)sim->T * sim->C * 4 * sim->N * 4, sim->stream)) != cudaSuccess) return e;
    sim->v_lazy = 0;
    return cudaSuccess;
}

cudaError_t launch_batched_reset(ranc_sim *sim, bool counters) {
    // Potentials and spike masks: the first tick reads v0 instead of V and
    // writes every spike mask, so nothing is written here (it also ignores
    // and rewrites the deferred idle ticks).
    sim->v_lazy = 1;
    sim->pend_dirty = 0;
    // The tick restarts at 0: the stamp clock moves to the next multiple of 16
    // past its current cycle, and no row holds bits after the clearing below.
    sim->sclock = (sim->sclock + 2 * kRows - 1) & ~(uint32_t)(kRows - 1);
    sim->all_active_ticks = 0;
    // Scheduler rows.  After normal stepping up to tick t, a row can hold
    // bits only if a delivery of tick t' < t targets a tick >= t, i.e. rows
    // t .. t + max_delay - 1 (mod 16): every other row was cleared when it was
    // read.  Only those rows are cleared, unless the rows may hold anything
    // (new handle, imported state, failed kernel).
    const size_t row = (size_t)sim->A * 16, block = row * kRows;  // bytes per row, per (tile, core)
    cudaError_t e;
    if (sim->ring_all_dirty || sim->max_delay >= kRows) {
        if ((e = cudaMemsetAsync(sim->ring, 0, (size_t)sim->T * sim->C * block, sim->stream)) != cudaSuccess) return e;
        sim->ring_all_dirty = 0;
    } else if (sim->max_delay > 0 && sim->tick > 0) {
        const int r0 = (int)(sim->tick & (kRows - 1)), n1 = std::min(sim->max_delay, kRows - r0), n2 = sim->max_delay - n1;
        uint8_t *base = reinterpret_cast<uint8_t *>(sim->ring);
        if ((e = cudaMemset2DAsync(base + r0 * row, block, 0, n1 * row, (size_t)sim->T * sim->C, sim->stream)) != cudaSuccess)
            return e;
        if (n2 > 0 && (e = cudaMemset2DAsync(base, block, 0, n2 * row, (size_t)sim->T * sim->C, sim->stream)) != cudaSuccess)
            return e;
    }
    if ((e = cudaMemsetAsync(sim->out, 0, (size_t)sim->B_pad * sim->n_outputs * 4, sim->stream)) != cudaSuccess) return e;
    if (counters && (e = cudaMemsetAsync(sim->cnt, 0, sim->cnt_len * 8, sim->stream)) != cudaSuccess) return e;
    if (counters && (e = cudaMemsetAsync(B_of(sim)->item_ticks, 0, 24, sim->stream)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Updated, deferred and active item-ticks since the last counter reset
// (synchronises the stream).
cudaError_t batched_item_ticks(ranc_sim *sim, unsigned long long *host3) {
    cudaError_t e = cudaMemcpyAsync(host3, B_of(sim)->item_ticks, 24, cudaMemcpyDeviceToHost, sim->stream);
    return e != cudaSuccess ? e : cudaStreamSynchronize(sim->stream);
}

// Makes the transposed-input buffer hold n_ticks ticks (may synchronise the
// stream and reallocate); *buffer receives its address.
cudaError_t batched_reserve_inputs(ranc_sim *sim, int n_ticks, const void **buffer) {
    Batched *bs = B_of(sim);
    const size_t need = (size_t)sim->T * n_ticks * bs->Lpad;  // uint4 units
    if (need > bs->inT_cap) {
        cudaError_t e = cudaStreamSynchronize(sim->stream);
        if (e != cudaSuccess) return e;
        if (bs->inT) cudaFree(bs->inT);
        bs->inT = nullptr;
        bs->inT_cap = 0;
        if (dev_alloc((void **)&bs->inT, need * 16) != cudaSuccess) return cudaErrorMemoryAllocation;
        bs->inT_cap = need;
    }
    if (buffer) *buffer = bs->inT;
    return cudaSuccess;
}

cudaError_t launch_batched_inputs(ranc_sim *sim, const uint32_t *dev_bits, int n_samples, int n_ticks) {
    Batched *bs = B_of(sim);
    cudaError_t er = batched_reserve_inputs(sim, n_ticks, nullptr);
    if (er != cudaSuccess) return er;
    const long long threads = (long long)sim->T * n_ticks * sim->in_words * 4 * 32;
    transpose_inputs<<<(unsigned)((threads + 255) / 256), 256, 0, sim->stream>>>(dev_bits, n_samples, n_ticks,
                                                                                sim->in_words, sim->T, (uint32_t *)bs->inT);
    sim->launches++;
    return cudaGetLastError();
}

cudaError_t launch_transpose_inputs(const uint32_t *x, int n_samples, int ticks, int words, int T, uint32_t *inT,
                                    cudaStream_t stream) {
    const long long threads = (long long)T * ticks * words * 4 * 32;
    if (threads == 0) return cudaSuccess;
    transpose_inputs<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(x, n_samples, ticks, words, T, inT);
    return cudaGetLastError();
}

cudaError_t launch_batched_export(ranc_sim *sim, int b0, int nb, int *v, uint32_t *spk, uint32_t *ring) {
    cudaError_t e0 = batched_materialize(sim);
    if (e0 != cudaSuccess) return e0;
    const long long total = (long long)nb * sim->C * sim->N + (long long)nb * sim->C * (sim->N / 32) +
                            (ring ? (long long)nb * sim->C * kRows * (sim->A / 32) : 0);
    if (sim->vmode == kVHalf)
        export_state<__half><<<(unsigned)grid_for(total), 256, 0, sim->stream>>>(
            (const __half *)sim->V, sim->spk, sim->ring, b0, nb, sim->C, sim->N, sim->A, v, spk, ring);
    else if (sim->vmode == kVInt16)
        export_state<int16_t><<<(unsigned)grid_for(total), 256, 0, sim->stream>>>(
            (const int16_t *)sim->V, sim->spk, sim->ring, b0, nb, sim->C, sim->N, sim->A, v, spk, ring);
    else
        export_state<int><<<(unsigned)grid_for(total), 256, 0, sim->stream>>>(
            (const int *)sim->V, sim->spk, sim->ring, b0, nb, sim->C, sim->N, sim->A, v, spk, ring);
    sim->launches++;
    return cudaGetLastError();
}

cudaError_t launch_batched_import(ranc_sim *sim, const int *v, const uint32_t *spk, const uint32_t *ring) {
    sim->v_lazy = 0;          // V and the spike masks are overwritten
    sim->ring_all_dirty = 1;  // any row may hold deliveries now
    sim->all_active_ticks = kRows;  // ... so every item is active until each row has been read once
    sim->pend_dirty = 0;
    if (cudaError_t e = cudaMemsetAsync(B_of(sim)->pend, 0, (size_t)2 * B_of(sim)->spitch, sim->stream); e != cudaSuccess)
        return e;
    const long long total = (long long)sim->B * sim->C * sim->N + (long long)sim->T * sim->C * 4 * sim->N +
                            (long long)sim->T * sim->C * kRows * sim->A * 4;
    if (sim->vmode == kVHalf)
        import_state<__half><<<(unsigned)grid_for(total), 256, 0, sim->stream>>>(
            (__half *)sim->V, sim->spk, sim->ring, sim->B, sim->T, sim->C, sim->N, sim->A, v, spk, ring);
    else if (sim->vmode == kVInt16)
        import_state<int16_t><<<(unsigned)grid_for(total), 256, 0, sim->stream>>>(
            (int16_t *)sim->V, sim->spk, sim->ring, sim->B, sim->T, sim->C, sim->N, sim->A, v, spk, ring);
    else
        import_state<int><<<(unsigned)grid_for(total), 256, 0, sim->stream>>>(
            (int *)sim->V, sim->spk, sim->ring, sim->B, sim->T, sim->C, sim->N, sim->A, v, spk, ring);
    sim->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free read of a sample range (see ranc_read_sample_state_noalloc).
// The canonical copies go to a fixed device array that every GPU loading this
// library holds until the process exits; no call allocates device memory.
// ---------------------------------------------------------------------------

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device`, looked up once per device
// with that device current (a host-side use of the symbol is not a device
// address).
cudaError_t noalloc_scratch(int device, void **ptr) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        int cur = 0;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        if (cur != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (cur != device) cudaSetDevice(cur);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = p;
    }
    *ptr = g_noalloc_ptr[device];
    return cudaSuccess;
}
}  // namespace

cudaError_t batched_export_noalloc(ranc_sim *sim, int b0, int nb, int *v_host, uint32_t *spk_host) {
    void *scratch = nullptr;
    cudaError_t e = noalloc_scratch(sim->device, &scratch);
    if (e != cudaSuccess) return e;
    const size_t per_v = (size_t)sim->C * sim->N, per_s = (size_t)sim->C * (sim->N / 32);
    int *v = static_cast<int *>(scratch);
    uint32_t *spk = reinterpret_cast<uint32_t *>(v + (size_t)nb * per_v);
    if ((e = launch_batched_export(sim, b0, nb, v, spk, nullptr)) != cudaSuccess) return e;
    if (v_host && (e = cudaMemcpyAsync(v_host, v, (size_t)nb * per_v * 4, cudaMemcpyDeviceToHost, sim->stream)) != cudaSuccess)
        return e;
    if (spk_host &&
        (e = cudaMemcpyAsync(spk_host, spk, (size_t)nb * per_s * 4, cudaMemcpyDeviceToHost, sim->stream)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

void batched_teardown(ranc_sim *sim) {
    Batched *bs = B_of(sim);
    if (!bs) return;
    void *ptrs[] = {bs->wfold, bs->fin_ptr, bs->fin_line, bs->outdeg, bs->inT, bs->stamp, bs->pend, bs->core_flags, bs->item_ticks};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete bs;
    sim->tmap = nullptr;
}

}  // namespace ranc
