// Batched path over several networks of different core shapes in one handle:
// one persistent launch per tick updates every core of every network (a
// design sweep simulated together; the paper motivates GPU simulation by the
// cost of sweeping RANC's configuration parameters, Sec. I and Sec. V).
//
// Per (network s, core c, sample tile j) work item, one tick of Alg. 1, as on
// the single-network batched path:
//   dV[n][m] = sum_a W[n][a] * S[m][a]        (Sec. II, Alg. 1 neuron block)
// with S the 0/1 active axons of the 128 samples of the tile and W[n][a] =
// w[type(a)][n] if axon a connects to neuron n (folded once at create; fp16
// operands and fp32 accumulation are exact, |partial sums| < 2^22), then
// leak, thresholds, reset, delivery into row (t + delay) mod 16 of the
// destination core of the same network (Sec. III-D) and output-bus counts.
//
// Shapes: axons A_s a multiple of 64 up to 512, neurons N_s a multiple of 128
// up to 512, any core count; one negative-threshold mode and one potential
// storage (the narrowest exact for every network) per handle.
//
// Pipeline of one CTA (640 threads, one CTA per SM, persistent over items):
//   all        the split: every item is classified active (its scheduler row
//              may hold bits, or input lines drive its core in this tick) or
//              idle (dV = 0: no operand, no MMA); the CTA takes its share of
//              the items by a cost prefix (cost per class and network shape)
//              computed in every CTA;
//   warps 0-15 workers: per item, (1) build the fp16 0/1 spike operand of an
//              active item from its scheduler row and input lines (row read
//              and cleared), (2) epilogue of the previous item, one 128-neuron
//              slice at a time: tensor memory -> registers, potential update,
//              32-sample spike masks, delivery, output bus, counters;
//   warp 16    tensor-memory allocation and MMA issue: per active item and
//              slice h, the K-blocks of 64 axons (4 MMAs of K = 16 each) into
//              one of four 128-column accumulators (a ring over the slices);
//   warp 17    weight loader: the folded weights of every (slice, K-block) of
//              the active items, 16 KB blocks stored pre-swizzled in global
//              memory, copied by the TMA engine (cp.async.bulk) into a ring of
//              weight stages ahead of the MMAs;
//   warp 18    prefetcher: the potentials (one contiguous block per item) and
//              the scheduler row of the items just ahead of the workers are
//              brought into L2 by bulk prefetches (cp.async.bulk.prefetch.L2),
//              so the epilogue's and the build's loads do not wait on HBM.
// Every mbarrier wait is bounded (global timer); a timeout sets the device
// error word and every role leaves its loop, drains the tensor core and the
// copies in flight, and frees tensor memory before the CTA exits.
//
// Layouts per network s (T tiles of 128 samples; item it = (core0_s + c) * T + j):
//   V     [T][C_s][4][N_s/32][P][32][E]  interleaved potentials as on the
//                                        single-network batched path
//   ring  [T][C_s][16][A_s][4]           word k of axon a = samples 32k..32k+31
//   spk   [T][C_s][4][N_s]               spike masks of the last tick
//   W     [C_s][N_s/128][A_s/64] blocks  128 neurons x 64 axons fp16, rows of
//                                        128 bytes with the 16-byte chunks
//                                        swizzled (chunk ^ row % 8)
// shared by all networks: inT [T][ticks][Lpad][4] input lines (sample-minor),
// stamp [16][items], out [B_pad][sum of output ids], cnt [T][cores][4].

#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "ranc_internal.cuh"
#include "ranc_ptx.cuh"
#include "ranc_tc.cuh"

namespace ranc {
namespace {

constexpr int kWorkersM = 16;                   // warps 0-15: operand build + epilogue
constexpr int kIssuerWarpM = 16;                // tensor memory, MMA issue
constexpr int kLoaderWarpM = 17;                // weight-block copies
constexpr int kPrefetchWarpM = 18;              // L2 prefetch of the items ahead of the workers
constexpr int kPrefetchAhead = 2;               // items prefetched ahead of the workers' epilogue
constexpr int kThreadsM = (kWorkersM + 4) * 32;  // warps 16-19 form one warpgroup
constexpr int kRegWorkerM = 104, kRegIssuerM = 48;
static_assert(kWorkersM * 32 * kRegWorkerM + 4 * 32 * kRegIssuerM <= kThreadsM * 96, "register split exceeds the launch");
constexpr uint32_t kBlk = 16384;  // one 16 KB block: 128 weight rows x 64 fp16, or 64 axons x 128 samples fp16
constexpr int kMaxKB = 8;         // axons <= 512
constexpr int kMaxStagesM = 6;
constexpr int kSlots = 4;         // accumulators of 128 tensor-memory columns (512 columns)
constexpr int kClsCapM = 16384;   // most items of a CTA whose classes are kept in shared memory
constexpr int kClsCapMinM = 8192; // fewest: a weight stage is dropped rather than the cache cut below this

// One network of a multi-network handle (device table).
struct SegDev {
    int C, A, N, NH, KB;    // cores, axons, neurons, N/128 slices, A/64 K-blocks
    int core0;              // first global core index
    long long voff;         // potentials: element offset of [T][C][4][N/32][P][32][E]
    long long roff;         // scheduler rows: word offset of [T][C][16][A][4]
    long long soff;         // spike masks: word offset of [T][C][4][N]
    long long poff;         // per-neuron arrays (prm, dst, v0): offset of [C][N]
    long long woff;         // weight blocks: offset of [C][NH][KB] (16 KB units)
    long long foff;         // fan-in offsets: offset of [C][A + 1]
    long long aoff;         // out-degrees: offset of [C][A]
    int cost_act, cost_idle;
};

struct MultiArgs {
    int n_seg, C, T, n_valid, Lpad, in_ticks, n_out, items, stages;
    long long tick;
    const SegDev *seg;         // [n_seg]
    const uint8_t *core_seg;   // [C] network of each global core
    const int4 *prm;           // {leak, pos_thr, neg_thr, reset} per neuron (by poff)
    const uint2 *dst;          // resolved destination per neuron: core within the network / global output id
    const int *v0;             // potentials at reset per neuron
    const int *fin_ptr, *fin_line;  // input lines driving (core, axon): fin_line[fin_ptr[a] .. fin_ptr[a + 1])
    const uint32_t *outdeg;    // connections of each (core, axon)
    const uint8_t *wblk;       // weight blocks (16 KB each)
    const uint4 *inT;
    int v0_now;                // first tick after a reset: V is v0 (not read)
    void *V;
    uint32_t *ring, *spk, *out;
    unsigned long long *cnt;   // [T][C][4]: spikes, packets, outputs, synaptic events
    int *err;
    const uint8_t *stamp_row;  // [items] stamps of this tick's scheduler row
    uint8_t *stamp;            // [16][spitch]
    long long spitch;
    uint32_t sclock;           // stamp clock of this tick
    int all_active;
    const uint8_t *core_flags; // [C] bit 0: some input line drives the core
    unsigned long long *item_ticks;  // [3 + 2 * n_seg]: updated, deferred (always 0 here), active item-ticks,
                                     // then updated and active item-ticks of each network
    int kbmax;                 // largest A/64 of the handle: operand blocks kept in shared memory
    int cls_cap;               // items of a CTA whose classes fit the shared-memory cache (at most kClsCapM)
    int stall_test;            // failure-detection tests only: CTA 0's issuer waits for its first weight
                               // block on a barrier armed with a transaction count no copy satisfies
    int dbg_plant;             // debug builds: site whose range checks fail on purpose (0: none)
};

// Split of the items over the CTAs by a cost prefix (as on the single-network
// path, without deferred items): CTA b takes the items whose exclusive prefix
// P satisfies b * W <= P * G < (b + 1) * W.  Run by all threads; on return
// cut_sh holds [i0, i1) and, when the range fits kClsCapM, cls_sm the class of
// each item of the range (2 active, 1 idle).  The prefix is formed per core
// (its T items share the network and the input flag; an input-driven core has
// all of them active), each thread over a contiguous run of cores; only the
// cores that hold a cut are walked item by item.  seg_sh (2 * n_seg counters)
// collects the per-network item counts of the CTA's range.
__device__ __noinline__ void split_multi(const MultiArgs &a, const int *cost_sh, long long *wsum_sh, int *cut_sh,
                                         uint8_t *cls_sm, unsigned *seg_sh) {
    const uint8_t *const stamp_row = a.stamp_row, *const core_flags = a.core_flags, *const core_seg = a.core_seg;
    const int C = a.C, T = a.T, n_seg = a.n_seg;
    const bool all_active = a.all_active != 0, inputs = a.tick < (long long)a.in_ticks;
    const uint8_t cycle = (uint8_t)(a.sclock >> 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 2 * n_seg; i += kThreadsM) seg_sh[i] = 0u;
    const int per = (C + kThreadsM - 1) / kThreadsM;
    const int g0 = min(C, tid * per), g1 = min(C, g0 + per);
    auto all_of = [&](int g) -> bool { return all_active || (inputs && (core_flags[g] & 1)); };
    auto n_active = [&](int g) -> int {  // active items of core g
        if (all_of(g)) return T;
        const uint8_t *st = stamp_row + (size_t)g * T;
        int n = 0;
        for (int j = 0; j < T; ++j) n += st[j] == cycle;
        return n;
    };
    long long csum = 0;
    for (int g = g0; g < g1; ++g) {
        const int s = core_seg[g], na = n_active(g);
        csum += (long long)na * cost_sh[2 * s] + (long long)(T - na) * cost_sh[2 * s + 1];
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
        for (int w = 0; w < kThreadsM / 32; ++w) {
            const long long x = wsum_sh[w];
            if (w < warp) P += x;
            W += x;
        }
        P += cinc - csum;
        const long long G = gridDim.x;
        const long long lo = ((long long)blockIdx.x * W + G - 1) / G, hi = ((long long)(blockIdx.x + 1) * W + G - 1) / G;
        int n0 = 0, n1 = 0;
        for (int g = g0; g < g1; ++g) {
            const int s = core_seg[g];
            const int ca = cost_sh[2 * s], ci = cost_sh[2 * s + 1];
            const bool all = all_of(g);
            const int na = all ? T : n_active(g);
            const long long cc = (long long)na * ca + (long long)(T - na) * ci;
            // items of this core whose exclusive prefix lies below lo / hi
            for (int b = 0; b < 2; ++b) {
                const long long lim = b ? hi : lo;
                int n = 0;
                if (P + cc <= lim) {
                    n = T;
                } else if (P < lim) {
                    long long Pj = P;
                    const uint8_t *st = stamp_row + (size_t)g * T;
                    for (int j = 0; j < T && Pj < lim; ++j, ++n) Pj += (all || st[j] == cycle) ? ca : ci;
                }
                (b ? n1 : n0) += n;
            }
            P += cc;
        }
        n0 = __reduce_add_sync(0xffffffffu, n0);
        n1 = __reduce_add_sync(0xffffffffu, n1);
        if (lane == 0 && (n0 | n1)) {
            atomicAdd(&cut_sh[0], n0);
            atomicAdd(&cut_sh[1], n1);
        }
    }
    __syncthreads();
    const int i0 = cut_sh[0], i1 = cut_sh[1], n_items = i1 - i0;
    int n_up = 0, n_act = 0;
    for (int li = tid; li < n_items; li += kThreadsM) {
        const int it = i0 + li, g = it / T;
        const bool act = all_of(g) || stamp_row[it] == cycle;
        if (n_items <= a.cls_cap) cls_sm[li] = act ? 2 : 1;
        const int s = core_seg[g];
        atomicAdd(&seg_sh[2 * s], 1u);
        if (act) atomicAdd(&seg_sh[2 * s + 1], 1u);
        ++n_up;
        n_act += act;
    }
    n_up = __reduce_add_sync(0xffffffffu, n_up);
    n_act = __reduce_add_sync(0xffffffffu, n_act);
    if (lane == 0 && n_up) atomicAdd(a.item_ticks, (unsigned long long)n_up);
    if (lane == 0 && n_act) atomicAdd(a.item_ticks + 2, (unsigned long long)n_act);
    __syncthreads();
    for (int s = tid; s < n_seg; s += kThreadsM) {
        if (seg_sh[2 * s]) atomicAdd(a.item_ticks + 3 + 2 * s, (unsigned long long)seg_sh[2 * s]);
        if (seg_sh[2 * s + 1]) atomicAdd(a.item_ticks + 4 + 2 * s, (unsigned long long)seg_sh[2 * s + 1]);
    }
}

template <typename VT, int kNegReset>
__global__ void __launch_bounds__(kThreadsM, 1) multi_tick_kernel(const __grid_constant__ MultiArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t s_full, s_free, acc_full[kSlots], acc_empty[kSlots], w_full[kMaxStagesM],
        w_empty[kMaxStagesM], bar_drain, bar_stall;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ volatile int cur_sh;  // item whose operand the workers build (prefetcher's position)
    __shared__ long long wsum_sh[kThreadsM / 32];
    __shared__ int cut_sh[2];
    __shared__ int cost_sh[2 * 256];
    __shared__ unsigned seg_sh[2 * 256];

    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = a.stages, T = a.T;
    uint8_t *Ssm = base;                                   // [kbmax] operand blocks
    uint8_t *Wsm = Ssm + (size_t)a.kbmax * kBlk;           // [S] weight stages
    uint2 *lut = reinterpret_cast<uint2 *>(Wsm + (size_t)S * kBlk);  // 16 x 8 B
    uint8_t *cls_sm = reinterpret_cast<uint8_t *>(lut) + 128;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = (int)(a.tick & (kRows - 1));

    if (tid < 16) {  // 4 fp16 values (1.0 or 0.0) per nibble of spike bits
        uint32_t w[2];
#pragma unroll
        for (int q = 0; q < 2; ++q)
            w[q] = (((tid >> (2 * q)) & 1) ? 0x3C00u : 0u) | (((tid >> (2 * q + 1)) & 1) ? 0x3C000000u : 0u);
        lut[tid] = make_uint2(w[0], w[1]);
    }
    for (int i = tid; i < a.n_seg; i += kThreadsM) {
        cost_sh[2 * i] = a.seg[i].cost_act;
        cost_sh[2 * i + 1] = a.seg[i].cost_idle;
    }
    if (tid == 0) {
        mbar_init(&s_full, kWorkersM);
        mbar_init(&s_free, 1);
        for (int k = 0; k < kSlots; ++k) {
            mbar_init(&acc_full[k], 1);
            mbar_init(&acc_empty[k], kWorkersM);
        }
        for (int k = 0; k < S; ++k) {
            mbar_init(&w_full[k], 1);
            mbar_init(&w_empty[k], 1);
        }
        mbar_init(&bar_drain, 1);
        mbar_init(&bar_stall, 1);
        abort_sh = 0;
        cur_sh = 0;
        cut_sh[0] = cut_sh[1] = 0;
        fence_mbar_init();
    }
    if (warp == kIssuerWarpM) tmem_alloc(&tmem_base_sh, 512);
    __syncthreads();
    split_multi(a, cost_sh, wsum_sh, cut_sh, cls_sm, seg_sh);
    const int i0 = cut_sh[0], i1 = cut_sh[1], n_items = i1 - i0;
    const bool cls_cached = n_items <= a.cls_cap;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const bool inputs = a.tick < (long long)a.in_ticks;
    const uint8_t cycle = (uint8_t)(a.sclock >> 4);
    auto active_at = [&](int li) -> bool {
        const int it = i0 + li;
        if (cls_cached) return cls_sm[li] == 2;
        return a.all_active || a.stamp_row[it] == cycle || (inputs && (a.core_flags[it / T] & 1));
    };
    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        if (abort_sh) return false;
        if (mbar_wait_bounded(bar, parity)) return true;
        abort_sh = 1;
        atomicExch(a.err, kErrTimeout);
        return false;
    };

    if (warp < kWorkersM) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kRegWorkerM) : "memory");
        // ------------------------------------------------------------ workers
        // Iteration k: build the operand of item k when it is active, then the
        // epilogue of item k - 1 (while the tensor core works on item k).
        // Epilogue unit of this warp in every slice h: TMEM lanes 32q..32q+31
        // (neuron h*128 + 32q + lane), samples 32cc .. 32cc+31 of the tile.
        const int q = warp & 3, cc = warp >> 2;
        constexpr int kVecs = 32 * (int)sizeof(VT) / 16;
        constexpr bool kHalf = std::is_same<VT, __half>::value;
        // With 2-byte potentials the loads of the epilogue's first slice are
        // issued before the build (their registers fit beside the build's).
        constexpr bool kPre0 = sizeof(VT) == 2;
        const int wt = warp * 32 + lane;  // build task index base: tasks wt and wt + 512 (2A <= 1024)
        int nb = 0;                       // operands built (phases of s_full / s_free)
        int ns = 0;                       // accumulator slices consumed (ring position)
        bool stop = false;
        // Words of the next active item's operand, loaded one build ahead (row
        // r0 receives no delivery in this tick: every delay is at least 1), and
        // the fan-in range, first input line and out-degree of each task's
        // axon, kept while the core does not change.
        int fg = -1, f0[2] = {0, 0}, f1[2] = {0, 0}, ln0[2] = {0, 0};
        uint32_t odr[2] = {0u, 0u};
        uint2 wr[2], wi[2];
        auto load_words = [&](int li) {
            const int it = i0 + li, g = it / T, j = it - g * T;
            const SegDev sd = a.seg[a.core_seg[g]];
            const int c = g - sd.core0;
            const uint2 *row = reinterpret_cast<const uint2 *>(a.ring + sd.roff + (((size_t)j * sd.C + c) * kRows + r0) * sd.A * 4);
            const bool newc = g != fg;
            fg = g;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int tau = wt + t * kWorkersM * 32, rax = tau >> 1, rhf = tau & 1;
                wr[t] = wi[t] = make_uint2(0u, 0u);
                if (tau >= 2 * sd.A) continue;
                wr[t] = row[rax * 2 + rhf];
                if (newc) {
                    odr[t] = a.outdeg[sd.aoff + (size_t)c * sd.A + rax];
                    if (inputs) {
                        const int *fp = a.fin_ptr + sd.foff + (size_t)c * (sd.A + 1) + rax;
                        f0[t] = fp[0];
                        f1[t] = fp[1];
                        ln0[t] = f1[t] > f0[t] ? a.fin_line[f0[t]] : 0;
                    }
                }
                if (inputs && f1[t] > f0[t]) {
                    const uint2 *in = reinterpret_cast<const uint2 *>(a.inT + ((size_t)j * a.in_ticks + a.tick) * a.Lpad) + rhf;
                    if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputLine, ln0[t], a.Lpad)) wi[t] = in[(size_t)ln0[t] * 2];
                    for (int e = f0[t] + 1; e < f1[t]; ++e) {  // further lines (each waits for its load)
                        const int ln = a.fin_line[e];
                        if (!RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputLine, ln, a.Lpad)) continue;
                        const uint2 y = in[(size_t)ln * 2];
                        wi[t].x |= y.x;
                        wi[t].y |= y.y;
                    }
                }
            }
        };
        auto next_active = [&](int li) {
            while (li < n_items && !active_at(li)) ++li;
            return li;
        };
        int kn = next_active(0);  // next item to build
        if (kn < n_items) load_words(kn);
        // One slice of the epilogue item as this lane sees it: parameters,
        // destination and 32 potentials of neuron h*128 + 32q + lane.
        struct Slice {
            int4 pr;
            uint2 dd;
            uint4 vb[kVecs];
        };
        auto load_slice = [&](const SegDev &sd, int ce, int je, int h, Slice &L) {
            const int n = h * 128 + q * 32 + lane;
            const size_t pn = (size_t)sd.poff + (size_t)ce * sd.N + n;
            L.pr = a.prm[pn];
            L.dd = a.dst[pn];
            if (a.v0_now) {
                const uint4 vz = v_splat<VT>(a.v0[pn]);
#pragma unroll
                for (int e = 0; e < kVecs; ++e) L.vb[e] = vz;
            } else {
                const uint4 *vp = reinterpret_cast<const uint4 *>(reinterpret_cast<const VT *>(a.V) + sd.voff +
                                                                  v_index<VT>(je, ce, cc, n & ~31, 0, sd.C, sd.N)) + lane;
#pragma unroll
                for (int e = 0; e < kVecs; ++e) L.vb[e] = vp[e * 32];
            }
        };
        for (int k = 0; k <= n_items && !stop; ++k) {
            if (warp == 0 && lane == 0) cur_sh = k;
            // ---- (0) slice 0 of the epilogue item k - 1: loads in flight during the build
            const int le = k - 1, ite = i0 + le, ge = ite / T, je = ite - ge * T;
            const SegDev sde = a.seg[a.core_seg[k > 0 ? ge : 0]];
            const int ce = ge - sde.core0;
            Slice cur;
            if (kPre0 && k > 0) load_slice(sde, ce, je, 0, cur);
            // ---- (1) build the operand of item k
            if (k < n_items && k == kn) {
                const int it = i0 + k, g = it / T, j = it - g * T;
                const SegDev sd = a.seg[a.core_seg[g]];
                const int c = g - sd.core0;
                if (!wait(&s_free, (nb & 1) ^ 1)) break;
                uint32_t ev = 0u;
                uint2 *row = reinterpret_cast<uint2 *>(a.ring + sd.roff + (((size_t)j * sd.C + c) * kRows + r0) * sd.A * 4);
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int tau = wt + t * kWorkersM * 32;
                    if (tau >= 2 * sd.A) continue;
                    const int rax = tau >> 1, rhf = tau & 1;
                    if (wr[t].x | wr[t].y) row[rax * 2 + rhf] = make_uint2(0u, 0u);
                    const uint2 w = make_uint2(wr[t].x | wi[t].x, wr[t].y | wi[t].y);
                    const int m0 = j * 128 + rhf * 64;
                    ev += odr[t] * (uint32_t)(__popc(w.x & valid_mask(a.n_valid, m0)) + __popc(w.y & valid_mask(a.n_valid, m0 + 32)));
                    // Row rax of the 64-sample half rhf (128-byte swizzle; the
                    // two halves write their chunks in opposite order).
                    const int r8 = rax & 7;
                    uint8_t *blk = Ssm + (size_t)(rax >> 6) * kBlk + ((rax & 63) >> 3) * 2048 + rhf * 1024 + r8 * 128;
#pragma unroll
                    for (int s8 = 0; s8 < 8; ++s8) {
                        const int chunk = s8 ^ (rhf * 4);
                        const uint32_t by = (chunk < 4 ? w.x : w.y) >> (8 * (chunk & 3));
                        const uint2 lo = lut[by & 0xFu], hi = lut[(by >> 4) & 0xFu];
                        *reinterpret_cast<uint4 *>(blk + ((chunk ^ r8) << 4)) = make_uint4(lo.x, lo.y, hi.x, hi.y);
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_full);
                ++nb;
                kn = next_active(k + 1);
                if (kn < n_items) load_words(kn);
                ev = __reduce_add_sync(0xffffffffu, ev);
                if (lane == 0 && ev) atomicAdd(a.cnt + ((size_t)j * a.C + g) * 4 + 3, (unsigned long long)ev);
            }
            // ---- (2) epilogue of item k - 1
            if (k == 0) continue;
            const bool act = active_at(le);
            VT *Vg = reinterpret_cast<VT *>(a.V) + sde.voff;
            const uint32_t valid = valid_mask(a.n_valid, je * 128 + cc * 32);
            uint32_t n_sp = 0, n_pk = 0, n_out = 0;
            for (int h = 0; h < sde.NH; ++h) {
                if (!kPre0 || h > 0) load_slice(sde, ce, je, h, cur);
                const int n = h * 128 + q * 32 + lane;
                const int4 pr = cur.pr;
                const uint2 dd = cur.dd;
                uint4 *vp = reinterpret_cast<uint4 *>(Vg + v_index<VT>(je, ce, cc, n & ~31, 0, sde.C, sde.N)) + lane;
                const int slot = ns & (kSlots - 1);
                if (act) {
                    if (!wait(&acc_full[slot], (ns / kSlots) & 1)) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                }
                uint32_t mask = 0u;
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    uint32_t d[16];
                    if (act) {
                        __syncwarp();
                        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(slot * 128 + cc * 32 + hf * 16), d);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) d[i] = 0u;  // no synaptic input: dV = 0.0f
                    }
                    if constexpr (kHalf) {
                        // Pairs of samples, exact as on the single-network path:
                        // V + leak in fp16, + dV in fp32, one monotone rounding,
                        // both thresholds and their predecessors representable.
                        const __half2 lam2 = __float2half2_rn((float)pr.x), pth2 = __float2half2_rn((float)pr.y),
                                      nth2 = __float2half2_rn((float)pr.z), r2 = __float2half2_rn((float)pr.w);
                        const uint32_t rst2 = *reinterpret_cast<const uint32_t *>(&r2);
                        uint32_t wv[8];
#pragma unroll
                        for (int q2 = 0; q2 < 2; ++q2) {
                            const uint4 u = cur.vb[hf * 2 + q2];
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
                            if constexpr (kNegReset) {
                                const uint32_t rm = fm | __hlt2_mask(x2, nth2);
                                wv[e] = (rm & rst2) | (~rm & *reinterpret_cast<const uint32_t *>(&x2));
                            } else {
                                const __half2 c2 = __hmax2(x2, nth2);
                                wv[e] = (fm & rst2) | (~fm & *reinterpret_cast<const uint32_t *>(&c2));
                            }
                            mask |= ((fm & 1u) | ((fm >> 15) & 2u)) << (hf * 16 + 2 * e);
                        }
                        vp[(hf * 2) * 32] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                        vp[(hf * 2 + 1) * 32] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
                    } else {
                        // Integer storage: dV + 1.5 * 2^23 in fp32 puts dV in the low
                        // mantissa bits; the bias is folded into the leak
                        // (wrap-around arithmetic, exact when V + dV + leak fits int32).
                        const uint32_t lam = (uint32_t)pr.x - 0x4B400000u;
                        int v[16];
                        unpack16<VT>(cur.vb, hf, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int x = (int)((uint32_t)v[i] + (uint32_t)f32_bits_minus_bias(d[i]) + lam);
                            const bool fire = x >= pr.y;
                            int y = kNegReset ? (x < pr.z ? pr.w : x) : max(x, pr.z);
                            v[i] = fire ? pr.w : y;
                            mask |= (fire ? 1u : 0u) << (hf * 16 + i);
                        }
                        store16<VT>(vp, hf, v);
                    }
                }
                if (act) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[slot]);
                    ++ns;
                }
                a.spk[sde.soff + (((size_t)je * sde.C + ce) * 4 + cc) * sde.N + n] = mask;
                const uint32_t live = mask & valid;
                const uint32_t kind = dest_kind(dd);
                n_sp += __popc(live);
                if (mask && kind == RANC_DEST_CORE && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestCore, dd.x, sde.C) &&
                    RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestAxon, dest_axon(dd), sde.A)) {
                    n_pk += __popc(live);
                    const uint32_t ax = dest_axon(dd);
                    const int r = (int)((a.tick + dest_delay(dd)) & (kRows - 1));
                    atomicOr(a.ring + sde.roff + ((((size_t)je * sde.C + dd.x) * kRows + r) * sde.A + ax) * 4 + cc, mask);
                    a.stamp[(size_t)r * a.spitch + (size_t)(sde.core0 + dd.x) * T + je] =
                        (uint8_t)((a.sclock + dest_delay(dd)) >> 4);
                }
                // Output bus: one warp-wide pass per output neuron that fired.
                uint32_t olanes = __ballot_sync(0xffffffffu, kind == RANC_DEST_OUTPUT && live != 0u);
                if (kind == RANC_DEST_OUTPUT) n_out += __popc(live);
                while (olanes) {
                    const int L = __ffs(olanes) - 1;
                    olanes &= olanes - 1u;
                    const uint32_t mL = __shfl_sync(0xffffffffu, live, L);
                    const uint32_t idL = __shfl_sync(0xffffffffu, dd.x, L);
                    if (((mL >> lane) & 1u) && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteOutputId, idL, a.n_out))
                        atomicAdd(a.out + (size_t)(je * 128 + cc * 32 + lane) * a.n_out + idL, 1u);
                }
            }
            if (stop) break;
            n_sp = __reduce_add_sync(0xffffffffu, n_sp);
            n_pk = __reduce_add_sync(0xffffffffu, n_pk);
            n_out = __reduce_add_sync(0xffffffffu, n_out);
            if (lane == 0 && (n_sp | n_pk | n_out)) {
                unsigned long long *cp = a.cnt + ((size_t)je * a.C + ge) * 4;
                atomicAdd(cp + 0, (unsigned long long)n_sp);
                atomicAdd(cp + 1, (unsigned long long)n_pk);
                atomicAdd(cp + 2, (unsigned long long)n_out);
            }
        }
    } else {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kRegIssuerM) : "memory");
        if (warp == kIssuerWarpM && lane == 0) {
            // ------------------------------------------------------------ MMA issuer
            int na = 0, ns = 0, nw = 0;  // operands consumed, accumulator slices, weight blocks
            for (int li = 0; li < n_items; ++li) {
                if (!active_at(li)) continue;
                const int it = i0 + li;
                const SegDev sd = a.seg[a.core_seg[it / T]];
                if (!wait(&s_full, na & 1)) break;
                tc_fence_after();
                bool ok = true;
                for (int h = 0; h < sd.NH && ok; ++h, ++ns) {
                    const int slot = ns & (kSlots - 1);
                    if (!(ok = wait(&acc_empty[slot], ((ns / kSlots) & 1) ^ 1))) break;
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(slot * 128);
                    for (int kb = 0; kb < sd.KB; ++kb, ++nw) {
                        const int st = nw % S;
                        uint64_t *wb = &w_full[st];
                        uint32_t wpar = (nw / S) & 1;
                        if (a.stall_test && blockIdx.x == 0 && nw == 0) {
                            // Failure-detection test: the wait for the first weight
                            // block is moved to a barrier that expects 16 bytes no
                            // copy delivers; it runs out (the block itself lands and
                            // the loader waits for it before exit).
                            mbar_arrive_expect_tx(&bar_stall, 16u);
                            wb = &bar_stall;
                            wpar = 0;
                        }
                        if (!(ok = wait(wb, wpar))) break;
                        tc_fence_after();
                        const uint32_t wa = smem_u32(Wsm + (size_t)st * kBlk), sb = smem_u32(Ssm + (size_t)kb * kBlk);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks)
                            mma_f16(d, smem_desc_kmajor(wa + ks * 32), smem_desc_mn(sb + ks * 4096), (kb | ks) != 0);
                        mma_commit(&w_empty[st]);
                    }
                    if (ok) mma_commit(&acc_full[slot]);
                }
                if (!ok) break;
                mma_commit(&s_free);
                ++na;
            }
            mma_commit(&bar_drain);  // every MMA issued completes before tensor memory is freed
            mbar_wait_bounded(&bar_drain, 0);
        } else if (warp == kLoaderWarpM && lane == 0) {
            // ------------------------------------------------------------ weight loader
            int nw = 0;  // blocks issued
            bool stalled = false;
            for (int li = 0; li < n_items && !stalled; ++li) {
                if (!active_at(li)) continue;
                const int it = i0 + li, g = it / T;
                const SegDev sd = a.seg[a.core_seg[g]];
                const uint8_t *src = a.wblk + ((size_t)sd.woff + (size_t)(g - sd.core0) * sd.NH * sd.KB) * kBlk;
                for (int b = 0; b < sd.NH * sd.KB; ++b, ++nw) {
                    const int st = nw % S;
                    if (!wait(&w_empty[st], ((nw / S) & 1) ^ 1)) {
                        stalled = true;
                        break;
                    }
                    mbar_arrive_expect_tx(&w_full[st], kBlk);
                    bulk_g2s(Wsm + (size_t)st * kBlk, src + (size_t)b * kBlk, kBlk, &w_full[st]);
                }
            }
            // Copies in flight land before the CTA exits: the last copy issued
            // on each stage completes its phase (bounded waits; a phase that
            // completed already passes at once).
            for (int k = 0; k < S; ++k) {
                const int idx = nw - 1 - k;
                if (idx < 0) break;
                mbar_wait_bounded(&w_full[idx % S], (idx / S) & 1);
            }
        } else if (warp == kPrefetchWarpM && lane == 0) {
            // ------------------------------------------------------------ prefetcher
            // Item li is prefetched once the workers have reached li - ahead
            // (polled with a bounded wait; no result depends on it).
            constexpr size_t kv = sizeof(VT);
            const unsigned long long t0 = global_ns();
            for (int li = 0; li < n_items && !abort_sh; ++li) {
                while (cur_sh + kPrefetchAhead < li && !abort_sh) {
                    if (global_ns() - t0 > 4 * kWaitLimitNs) break;
                    __nanosleep(200);
                }
                const int it = i0 + li, g = it / T, j = it - g * T;
                const SegDev sd = a.seg[a.core_seg[g]];
                const int c = g - sd.core0;
                if (!a.v0_now)
                    prefetch_l2(reinterpret_cast<const uint8_t *>(a.V) +
                                    (sd.voff + v_index<VT>(j, c, 0, 0, 0, sd.C, sd.N)) * kv,
                                (uint32_t)(128 * sd.N * kv));
                if (active_at(li))
                    prefetch_l2(a.ring + sd.roff + (((size_t)j * sd.C + c) * kRows + r0) * sd.A * 4, (uint32_t)sd.A * 16u);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kIssuerWarpM) tmem_dealloc(tmem, 512);
}

// Canonical copies of samples [b0, b0 + nb): v [nb][P] and spk [nb][P/32],
// P = sum over the networks of C_s * N_s (network s's cores at offset poff_s,
// core-major, neuron-minor); with v0_now the state is the reset state.
template <typename VT>
__global__ void export_multi(const SegDev *seg, int n_seg, const VT *V, const uint32_t *spkb, const int *v0, int v0_now,
                             int b0, int nb, long long P, int *v, uint32_t *spk) {
    const long long nv = (long long)nb * P, ns = nv / 32;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nv + ns; f += (long long)gridDim.x * blockDim.x) {
        const bool is_v = f < nv;
        const long long g = is_v ? f : (f - nv) * 32;  // first neuron of the spike word
        const int b = b0 + (int)(g / P);
        const long long r = g % P;
        int lo = 0, hi = n_seg - 1;  // network holding canonical offset r
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg[mid].poff <= r) lo = mid;
            else hi = mid - 1;
        }
        const SegDev &sd = seg[lo];
        const int c = (int)((r - sd.poff) / sd.N), n = (int)((r - sd.poff) % sd.N);
        const int j = b >> 7, cc = (b & 127) >> 5, i = b & 31;
        if (is_v) {
            v[f] = v0_now ? v0[sd.poff + (long long)c * sd.N + n]
                          : v_to_int<VT>(V[sd.voff + v_index<VT>(j, c, cc, n, i, sd.C, sd.N)]);
        } else {
            uint32_t word = 0u;
            if (!v0_now)
                for (int k = 0; k < 32; ++k)
                    word |= ((spkb[sd.soff + (((long long)j * sd.C + c) * 4 + cc) * sd.N + n + k] >> i) & 1u) << k;
            spk[f - nv] = word;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct Multi {
    int n_seg = 0, kbmax = 0, stages = 4, n_sm = 0, Lpad = 0;
    // Split cost of an item that receives spikes: cost_item + cost_slice per
    // slice + cost_mma per (K-block, slice) MMA group; of one that receives
    // none: 2 * cost_slice per slice.  The defaults are a least-squares fit of
    // per-CTA busy times against the CTAs' item mix on a 64-network sweep
    // (units of about 0.4 us: 1.55 us per item, 1.2 us per slice, 0.4 us per
    // MMA group; 2.5 us per slice of an idle item, whose potential loads find
    // no operand build to hide behind).
    int cost_item = 4, cost_mma = 1, cost_slice = 3;
    size_t smem = 0;
    std::vector<SegDev> seg;          // host copy of the network table
    SegDev *seg_dev = nullptr;
    uint8_t *core_seg = nullptr, *core_flags = nullptr, *wblk = nullptr, *stamp = nullptr;
    int *fin_ptr = nullptr, *fin_line = nullptr;
    uint32_t *outdeg = nullptr;
    uint4 *inT = nullptr;
    size_t inT_cap = 0;
    unsigned long long *item_ticks = nullptr;  // [3 + 2 * n_seg]
    long long spitch = 0, ring_words = 0, v_elems = 0, spk_words = 0;
    std::vector<int> max_delay;       // per network: largest core-to-core delay
};

// Split costs of network sd's items (int32: at most 1024 + 1024 * 8 * 4 + 1024 * 4 per item).
void set_costs(SegDev &sd, const Multi &m) {
    sd.cost_act = std::max(1, m.cost_item + m.cost_mma * sd.KB * sd.NH + m.cost_slice * sd.NH);
    sd.cost_idle = std::max(1, 2 * m.cost_slice * sd.NH);
}

Multi *M_of(ranc_sim *s) { return static_cast<Multi *>(s->multi); }

long long grid_m(long long n) { return std::max<long long>(1, std::min<long long>((n + 255) / 256, 8192)); }

// Shared memory of a CTA: the operand blocks and weight stages, the table
// and the class cache, whose capacity takes what is left of 227 KB less
// 5 KB for the kernel's static shared memory (4.4 KB), at most kClsCapM.
// (The kernel's shared-memory attribute is raised to the largest of these at
// create, which fails cleanly if static + dynamic ever exceeded 227 KB.)
constexpr long long kSmemBudgetM = 227 * 1024 - 5 * 1024;
int cls_cap_for(int kbmax, int stages) {
    const long long left = kSmemBudgetM - (1024 + (long long)(kbmax + stages) * kBlk + 128);
    return (int)std::max(0LL, std::min<long long>(kClsCapM, left) & ~15LL);
}
size_t smem_for(int kbmax, int stages) { return 1024 + (size_t)(kbmax + stages) * kBlk + 128 + cls_cap_for(kbmax, stages); }

template <typename VT, int kNR>
cudaError_t raise_multi_smem(size_t bytes) {
    return raise_smem_limit((const void *)multi_tick_kernel<VT, kNR>, (int)bytes);
}

}  // namespace

bool multi_shape_ok(int A, int N) { return A % 64 == 0 && A >= 64 && A <= 64 * kMaxKB && N % 128 == 0 && N >= 128 && N <= 512; }

int multi_max_stages(int kbmax) {
    int s = kMaxStagesM;
    while (s > 2 && cls_cap_for(kbmax, s) < kClsCapMinM) --s;
    return s;
}

cudaError_t multi_setup(ranc_sim *sim, const ranc_desc *const *descs, int n, std::string &why) {
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
    Multi *m = new (std::nothrow) Multi();
    if (!m) {
        why = "host allocation";
        return cudaErrorMemoryAllocation;
    }
    sim->multi = m;
    m->n_seg = n;
    m->n_sm = prop.multiProcessorCount;
    m->Lpad = sim->in_words * 32;
    sim->T = (sim->B + kTileS - 1) / kTileS;
    sim->B_pad = sim->T * kTileS;
    const int T = sim->T;

    // Potential storage: the narrowest format that is exact for every network
    // (kVInt32 < kVInt16 < kVHalf: the smallest code of the networks).
    int vmode = kVHalf;
    int C_total = 0;
    long long P = 0, vsz_elems = 0, ring_w = 0, spk_w = 0, wblocks = 0, fptr_n = 0, aout_n = 0;
    m->seg.resize(n);
    m->max_delay.assign(n, 0);
    for (int s = 0; s < n; s++) {
        const ranc_desc *d = descs[s];
        const int C = d->n_cores, A = d->axons, N = d->neurons;
        vmode = std::min(vmode, potential_format_of(d));
        for (size_t i = 0; i < (size_t)C * N; i++)
            if (d->dest[i].kind == RANC_DEST_CORE) m->max_delay[s] = std::max<int>(m->max_delay[s], d->dest[i].delay);
        SegDev &sd = m->seg[s];
        sd.C = C; sd.A = A; sd.N = N; sd.NH = N / 128; sd.KB = A / 64; sd.core0 = C_total;
        sd.voff = vsz_elems; sd.roff = ring_w; sd.soff = spk_w; sd.poff = P; sd.woff = wblocks; sd.foff = fptr_n;
        sd.aoff = aout_n;
        set_costs(sd, *m);
        C_total += C;
        vsz_elems += (long long)T * C * 4 * N * 32;
        ring_w += (long long)T * C * kRows * A * 4;
        spk_w += (long long)T * C * 4 * N;
        P += (long long)C * N;
        wblocks += (long long)C * sd.NH * sd.KB;
        fptr_n += (long long)C * (A + 1);
        aout_n += (long long)C * A;
        m->kbmax = std::max(m->kbmax, sd.KB);
    }
    sim->vmode = vmode;
    sim->max_delay = 0;
    for (int s = 0; s < n; s++) sim->max_delay = std::max(sim->max_delay, m->max_delay[s]);
    m->stages = std::min(4, multi_max_stages(m->kbmax));
    m->smem = smem_for(m->kbmax, multi_max_stages(m->kbmax));
    m->ring_words = ring_w;
    m->v_elems = vsz_elems;
    m->spk_words = spk_w;
    m->spitch = ((long long)T * C_total + 127) / 128 * 128;

    // Host arrays: per-neuron parameters and destinations (output ids moved
    // by the ids of the networks before), folded and pre-swizzled weights,
    // input fan-in per (core, axon), out-degrees, per-core flags.
    std::vector<int4> prm((size_t)P);
    std::vector<uint2> dst((size_t)P);
    std::vector<int> v0((size_t)P);
    std::vector<int> fptr((size_t)fptr_n), fline;
    std::vector<uint32_t> od((size_t)aout_n, 0u);
    std::vector<uint8_t> cseg(C_total), cfl(C_total, 0);
    std::vector<uint16_t> wb((size_t)wblocks * (kBlk / 2));
    int out0 = 0;
    for (int s = 0; s < n; s++) {
        const ranc_desc *d = descs[s];
        const SegDev &sd = m->seg[s];
        const int C = sd.C, A = sd.A, N = sd.N, K = d->n_types, NWd = N / 32;
        std::vector<int> core_at((size_t)d->grid_w * d->grid_h, -1);
        for (int c = 0; c < C; c++) core_at[(size_t)d->core_xy[2 * c + 1] * d->grid_w + d->core_xy[2 * c]] = c;
        for (int c = 0; c < C; c++) {
            cseg[sd.core0 + c] = (uint8_t)s;
            for (int nn = 0; nn < N; nn++) {
                const size_t i = (size_t)c * N + nn, o = (size_t)sd.poff + i;
                prm[o] = make_int4(d->leak[i], d->pos_thr[i], d->neg_thr[i], d->reset[i]);
                v0[o] = d->v0[i];
                const ranc_dest &t = d->dest[i];
                uint32_t target = 0;
                if (t.kind == RANC_DEST_CORE)
                    target = (uint32_t)core_at[(size_t)(d->core_xy[2 * c + 1] + t.dy) * d->grid_w + (d->core_xy[2 * c] + t.dx)];
                else if (t.kind == RANC_DEST_OUTPUT)
                    target = (uint32_t)(out0 + t.axon);
                dst[o] = make_uint2(target, (uint32_t)t.axon | ((uint32_t)t.delay << 16) | ((uint32_t)t.kind << 24));
            }
            // Folded weights of core c: block (h, kb) holds neurons 128h.. x axons
            // 64kb.., row r = neuron, 16-byte chunk q of the row at q ^ (r % 8).
            for (int ax = 0; ax < A; ax++) {
                const uint32_t *row = d->crossbar + ((size_t)c * A + ax) * NWd;
                const int k = d->axon_type[(size_t)c * A + ax];
                const int kb = ax >> 6, q16 = (ax & 63) >> 3, e8 = ax & 7;
                const int16_t *wrow = d->weight + ((size_t)c * K + k) * N;
                for (int wd = 0; wd < NWd; wd++) {  // the connections of this axon, word by word
                    uint32_t bits = row[wd];
                    od[(size_t)sd.aoff + (size_t)c * A + ax] += (uint32_t)__builtin_popcount(bits);
                    while (bits) {
                        const int nn = wd * 32 + __builtin_ctz(bits);
                        bits &= bits - 1u;
                        const int h = nn >> 7, r = nn & 127;
                        const size_t blk = (size_t)sd.woff + ((size_t)c * sd.NH + h) * sd.KB + kb;
                        const __half hv = __float2half((float)wrow[nn]);
                        wb[blk * (kBlk / 2) + (size_t)r * 64 + ((q16 ^ (r & 7)) << 3) + e8] =
                            *reinterpret_cast<const uint16_t *>(&hv);
                    }
                }
            }
        }
        // Input fan-in of every (core, axon) of this network.
        std::vector<std::vector<int>> lists((size_t)C * A);
        for (int i = 0; i < d->n_inputs; i++)
            for (int k = d->in_offsets[i]; k < d->in_offsets[i + 1]; k++)
                lists[(size_t)d->in_core[k] * A + d->in_axon[k]].push_back(i);
        for (int c = 0; c < C; c++) {
            bool driven = false;
            for (int ax = 0; ax < A; ax++) {
                fptr[(size_t)sd.foff + (size_t)c * (A + 1) + ax] = (int)fline.size();
                for (int L : lists[(size_t)c * A + ax]) fline.push_back(L);
                driven = driven || !lists[(size_t)c * A + ax].empty();
            }
            fptr[(size_t)sd.foff + (size_t)c * (A + 1) + A] = (int)fline.size();
            cfl[sd.core0 + c] = driven ? 1 : 0;
        }
        out0 += d->n_outputs;
    }
    if (fline.empty()) fline.push_back(0);

    const size_t vsz = sim->vmode == kVInt32 ? 4 : 2;
    if (dev_alloc((void **)&m->seg_dev, sizeof(SegDev) * n) != cudaSuccess ||
        dev_alloc((void **)&m->core_seg, C_total) != cudaSuccess || dev_alloc((void **)&m->core_flags, C_total) != cudaSuccess ||
        dev_alloc((void **)&m->wblk, wb.size() * 2) != cudaSuccess ||
        dev_alloc((void **)&m->fin_ptr, fptr.size() * 4) != cudaSuccess ||
        dev_alloc((void **)&m->fin_line, fline.size() * 4) != cudaSuccess ||
        dev_alloc((void **)&m->outdeg, od.size() * 4) != cudaSuccess ||
        dev_alloc((void **)&sim->prm, prm.size() * sizeof(int4)) != cudaSuccess ||
        dev_alloc((void **)&sim->dst, dst.size() * sizeof(uint2)) != cudaSuccess ||
        dev_alloc((void **)&sim->v0, v0.size() * 4) != cudaSuccess ||
        dev_alloc((void **)&sim->V, (size_t)vsz_elems * vsz) != cudaSuccess ||
        dev_alloc((void **)&sim->ring, (size_t)ring_w * 4) != cudaSuccess ||
        dev_alloc((void **)&sim->spk, (size_t)spk_w * 4) != cudaSuccess ||
        dev_alloc((void **)&sim->out, (size_t)sim->B_pad * sim->n_outputs * 4) != cudaSuccess ||
        dev_alloc((void **)&sim->cnt, (size_t)T * C_total * 4 * 8) != cudaSuccess ||
        dev_alloc((void **)&m->stamp, (size_t)kRows * m->spitch) != cudaSuccess ||
        dev_alloc((void **)&m->item_ticks, (3 + 2 * (size_t)n) * 8) != cudaSuccess) {
        why = "device allocation of the multi-network state failed";
        return cudaErrorMemoryAllocation;
    }
    sim->cnt_len = (size_t)T * C_total * 4;
    if ((e = cudaMemcpy(m->seg_dev, m->seg.data(), sizeof(SegDev) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->core_seg, cseg.data(), C_total, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->core_flags, cfl.data(), C_total, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->wblk, wb.data(), wb.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->fin_ptr, fptr.data(), fptr.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->fin_line, fline.data(), fline.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(m->outdeg, od.data(), od.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(sim->prm, prm.data(), prm.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(sim->dst, dst.data(), dst.size() * sizeof(uint2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(sim->v0, v0.data(), v0.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(m->stamp, 0, (size_t)kRows * m->spitch)) != cudaSuccess ||
        (e = cudaMemset(m->item_ticks, 0, (3 + 2 * (size_t)n) * 8)) != cudaSuccess) {
        why = "copy of the multi-network arrays";
        return e;
    }
    sim->nps = P;
    sim->C = C_total;
    const size_t sm = m->smem;
    if ((e = raise_multi_smem<__half, 0>(sm)) != cudaSuccess || (e = raise_multi_smem<__half, 1>(sm)) != cudaSuccess ||
        (e = raise_multi_smem<int16_t, 0>(sm)) != cudaSuccess || (e = raise_multi_smem<int16_t, 1>(sm)) != cudaSuccess ||
        (e = raise_multi_smem<int, 0>(sm)) != cudaSuccess || (e = raise_multi_smem<int, 1>(sm)) != cudaSuccess)
        why = "kernel shared-memory attribute";
    return e;
}

cudaError_t launch_multi_tick(ranc_sim *sim) {
    Multi *m = M_of(sim);
    MultiArgs a{};
    a.n_seg = m->n_seg; a.C = sim->C; a.T = sim->T; a.n_valid = sim->n_valid; a.Lpad = m->Lpad;
    a.in_ticks = m->inT ? sim->in_ticks : 0; a.n_out = sim->n_outputs; a.items = sim->T * sim->C; a.stages = m->stages;
    a.tick = sim->tick; a.seg = m->seg_dev; a.core_seg = m->core_seg; a.prm = sim->prm; a.dst = sim->dst; a.v0 = sim->v0;
    a.fin_ptr = m->fin_ptr; a.fin_line = m->fin_line; a.outdeg = m->outdeg; a.wblk = m->wblk; a.inT = m->inT;
    a.v0_now = sim->v_lazy; a.V = sim->V; a.ring = sim->ring; a.spk = sim->spk; a.out = sim->out; a.cnt = sim->cnt;
    a.err = sim->err;
    if (((sim->sclock ^ (uint32_t)sim->tick) & (kRows - 1)) != 0) {  // as on the single-network path
        sim->sclock = ((sim->sclock + 2 * kRows) & ~(uint32_t)(kRows - 1)) | ((uint32_t)sim->tick & (kRows - 1));
        sim->all_active_ticks = kRows;
    }
    a.stamp = m->stamp; a.spitch = m->spitch; a.stamp_row = m->stamp + (size_t)(sim->tick & (kRows - 1)) * m->spitch;
    a.sclock = sim->sclock; a.all_active = sim->all_active_ticks > 0; a.core_flags = m->core_flags;
    a.item_ticks = m->item_ticks; a.kbmax = m->kbmax; a.cls_cap = cls_cap_for(m->kbmax, m->stages); a.stall_test = sim->stall_test; a.dbg_plant = sim->dbg_plant;
    const int grid = std::min(m->n_sm, a.items);
    const size_t smem = smem_for(m->kbmax, m->stages);
    auto kern = sim->vmode == kVHalf    ? (sim->neg_mode ? multi_tick_kernel<__half, 1> : multi_tick_kernel<__half, 0>)
                : sim->vmode == kVInt16 ? (sim->neg_mode ? multi_tick_kernel<int16_t, 1> : multi_tick_kernel<int16_t, 0>)
                                        : (sim->neg_mode ? multi_tick_kernel<int, 1> : multi_tick_kernel<int, 0>);
    kern<<<grid, kThreadsM, smem, sim->stream>>>(a);
    sim->v_lazy = 0;
    sim->sclock++;
    if (sim->all_active_ticks > 0) --sim->all_active_ticks;
    return cudaGetLastError();
}

cudaError_t launch_multi_reset(ranc_sim *sim, bool counters) {
    Multi *m = M_of(sim);
    sim->v_lazy = 1;  // the first tick reads v0 and writes every spike mask
    sim->sclock = (sim->sclock + 2 * kRows - 1) & ~(uint32_t)(kRows - 1);
    sim->all_active_ticks = 0;
    cudaError_t e;
    if (sim->ring_all_dirty) {
        if ((e = cudaMemsetAsync(sim->ring, 0, (size_t)m->ring_words * 4, sim->stream)) != cudaSuccess) return e;
        sim->ring_all_dirty = 0;
    } else if (sim->tick > 0) {
        // Rows tick .. tick + d_max - 1 (mod 16) of every (tile, core) of each
        // network can still hold deliveries; every other row was cleared when read.
        for (int s = 0; s < m->n_seg; s++) {
            const SegDev &sd = m->seg[s];
            const int dmax = m->max_delay[s];
            if (dmax == 0) continue;
            const size_t row = (size_t)sd.A * 16, block = row * kRows;
            uint8_t *base = reinterpret_cast<uint8_t *>(sim->ring + sd.roff);
            const int r0 = (int)(sim->tick & (kRows - 1)), n1 = std::min(dmax, kRows - r0), n2 = dmax - n1;
            if ((e = cudaMemset2DAsync(base + r0 * row, block, 0, n1 * row, (size_t)sim->T * sd.C, sim->stream)) != cudaSuccess)
                return e;
            if (n2 > 0 && (e = cudaMemset2DAsync(base, block, 0, n2 * row, (size_t)sim->T * sd.C, sim->stream)) != cudaSuccess)
                return e;
        }
    }
    if ((e = cudaMemsetAsync(sim->out, 0, (size_t)sim->B_pad * sim->n_outputs * 4, sim->stream)) != cudaSuccess) return e;
    if (counters && (e = cudaMemsetAsync(sim->cnt, 0, sim->cnt_len * 8, sim->stream)) != cudaSuccess) return e;
    if (counters && (e = cudaMemsetAsync(m->item_ticks, 0, (3 + 2 * (size_t)m->n_seg) * 8, sim->stream)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t multi_item_ticks(ranc_sim *sim, unsigned long long *host3) {
    cudaError_t e = cudaMemcpyAsync(host3, M_of(sim)->item_ticks, 24, cudaMemcpyDeviceToHost, sim->stream);
    return e != cudaSuccess ? e : cudaStreamSynchronize(sim->stream);
}

cudaError_t multi_network_items(ranc_sim *sim, int k, unsigned long long *host2) {
    cudaError_t e = cudaMemcpyAsync(host2, M_of(sim)->item_ticks + 3 + 2 * (size_t)k, 16, cudaMemcpyDeviceToHost, sim->stream);
    return e != cudaSuccess ? e : cudaStreamSynchronize(sim->stream);
}

int multi_networks(const ranc_sim *sim) { return static_cast<const Multi *>(sim->multi)->n_seg; }

cudaError_t multi_reserve_inputs(ranc_sim *sim, int n_ticks, const void **buffer) {
    Multi *m = M_of(sim);
    const size_t need = (size_t)sim->T * n_ticks * m->Lpad;  // uint4 units
    if (need > m->inT_cap) {
        cudaError_t e = cudaStreamSynchronize(sim->stream);
        if (e != cudaSuccess) return e;
        if (m->inT) cudaFree(m->inT);
        m->inT = nullptr;
        m->inT_cap = 0;
        if (dev_alloc((void **)&m->inT, need * 16) != cudaSuccess) return cudaErrorMemoryAllocation;
        m->inT_cap = need;
    }
    if (buffer) *buffer = m->inT;
    return cudaSuccess;
}

cudaError_t launch_multi_inputs(ranc_sim *sim, const uint32_t *dev_bits, int n_samples, int n_ticks) {
    Multi *m = M_of(sim);
    cudaError_t e = multi_reserve_inputs(sim, n_ticks, nullptr);
    if (e != cudaSuccess) return e;
    e = launch_transpose_inputs(dev_bits, n_samples, n_ticks, sim->in_words, sim->T, (uint32_t *)m->inT, sim->stream);
    sim->launches++;
    return e;
}

cudaError_t launch_multi_export(ranc_sim *sim, int b0, int nb, int *v, uint32_t *spk) {
    Multi *m = M_of(sim);
    const long long total = (long long)nb * sim->nps + (long long)nb * sim->nps / 32;
    const unsigned g = (unsigned)grid_m(total);
    if (sim->vmode == kVHalf)
        export_multi<__half><<<g, 256, 0, sim->stream>>>(m->seg_dev, m->n_seg, (const __half *)sim->V, sim->spk, sim->v0,
                                                         sim->v_lazy, b0, nb, sim->nps, v, spk);
    else if (sim->vmode == kVInt16)
        export_multi<int16_t><<<g, 256, 0, sim->stream>>>(m->seg_dev, m->n_seg, (const int16_t *)sim->V, sim->spk, sim->v0,
                                                          sim->v_lazy, b0, nb, sim->nps, v, spk);
    else
        export_multi<int><<<g, 256, 0, sim->stream>>>(m->seg_dev, m->n_seg, (const int *)sim->V, sim->spk, sim->v0,
                                                      sim->v_lazy, b0, nb, sim->nps, v, spk);
    sim->launches++;
    return cudaGetLastError();
}

void multi_get_tuning(const ranc_sim *sim, int *stages, int *max_stages, int *cost_item, int *cost_mma, int *cost_slice) {
    const Multi *m = static_cast<const Multi *>(sim->multi);
    *stages = m->stages;
    *max_stages = multi_max_stages(m->kbmax);
    *cost_item = m->cost_item;
    *cost_mma = m->cost_mma;
    *cost_slice = m->cost_slice;
}

cudaError_t multi_set_tuning(ranc_sim *sim, int stages, int cost_item, int cost_mma, int cost_slice) {
    Multi *m = M_of(sim);
    m->stages = stages;
    m->cost_item = cost_item;
    m->cost_mma = cost_mma;
    m->cost_slice = cost_slice;
    for (SegDev &sd : m->seg) set_costs(sd, *m);
    cudaError_t e = cudaMemcpyAsync(m->seg_dev, m->seg.data(), sizeof(SegDev) * m->n_seg, cudaMemcpyHostToDevice, sim->stream);
    return e != cudaSuccess ? e : cudaStreamSynchronize(sim->stream);
}

void multi_teardown(ranc_sim *sim) {
    Multi *m = M_of(sim);
    if (!m) return;
    void *ptrs[] = {m->seg_dev, m->core_seg, m->core_flags, m->wblk, m->stamp, m->fin_ptr, m->fin_line, m->outdeg, m->inT,
                    m->item_ticks};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete m;
    sim->multi = nullptr;
}

}  // namespace ranc
