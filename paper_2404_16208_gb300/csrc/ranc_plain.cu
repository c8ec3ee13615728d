// Plain path: one CTA per (core, sample), one thread per neuron.
//
// One launch is one tick of Alg. 1 for every core of every sample:
//   1. scheduler row (tick mod 16) read and cleared (Sec. III-E);
//   2. input lines of this tick ORed into that row (Alg. 1, packets of the
//      current tick);
//   3. crossbar integration (Alg. 1 neuron block; Sec. III-C): the core's
//      bit-packed crossbar is staged into shared memory by one bulk copy of
//      the TMA engine, overlapped with steps 1-2; each neuron ANDs the active
//      axon bits with its row of connection bits and counts, per axon type,
//      the surviving bits with popc, so dV = sum_k w[k] * count_k;
//   4. leak, positive / negative threshold and reset;
//   5. spikes compacted with one warp ballot per 32 neurons; kind-core spikes
//      delivered with atomicOr into row (tick + delay) mod 16 of the
//      destination scheduler (Sec. III-D), kind-output spikes counted on the
//      output bus.
// Rows written at tick t are t+1..t+15 (mod 16), never the row being read, so
// the launch has no read/write race; OR and integer addition are order
// independent, so the result does not depend on scheduling.

#include <algorithm>

#include "ranc_internal.cuh"
#include "ranc_ptx.cuh"

namespace ranc {

// Weight of type k from a neuron's 8 packed int16 weights (selects, no
// indexed register array).
__device__ __forceinline__ int weight_of(const uint32_t (&wr)[4], int k) {
    const uint32_t lo = (k & 2) ? wr[1] : wr[0], hi = (k & 2) ? wr[3] : wr[2];
    return (int)(int16_t)(((k & 4) ? hi : lo) >> (16 * (k & 1)));
}

// Active axons of `ncores` cores in type-sorted order: bit p of core j's SW
// sorted words is bit perm[j * SW * 32 + p] of its AW words in original order
// (0 for a position without axon).  Thread t of nt (a multiple of 32) takes
// positions t, t + nt, ...; the lanes of a warp hold 32 consecutive positions
// of one word, so one ballot builds it.
__device__ __forceinline__ void gather_sorted(const uint32_t *s, const uint16_t *perm, int AW, int SW, int ncores,
                                              uint32_t *sp, int t, int nt) {
    const int P = SW * 32;
    for (int i = t; i < ncores * P; i += nt) {
        const int j = i / P, ia = perm[i];
        const bool on = ia != 0xFFFF && ((s[j * AW + (ia >> 5)] >> (ia & 31)) & 1u);
        const unsigned word = __ballot_sync(0xffffffffu, on);
        if ((i & 31) == 0) sp[i >> 5] = word;
    }
}

// dV and the synaptic-event count of one neuron over the sorted active axons
// sp: every sorted word holds one type, so a word costs one popc.
__device__ __forceinline__ int integrate_sorted(const uint32_t *sp, const uint32_t *xr, int N, const int8_t *wt, int SW,
                                                const uint32_t (&wr)[4], uint32_t &syn) {
    int dv = 0;
    for (int w = 0; w < SW; ++w) {
        const uint32_t sw = sp[w];
        if (sw == 0u) continue;  // uniform across the core's threads
        const uint32_t c1 = __popc(sw & xr[(size_t)w * N]);
        syn += c1;
        dv += weight_of(wr, wt[w]) * (int)c1;
    }
    return dv;
}

// The same with the sorted words grouped by type: tb[k] .. tb[k+1] are the
// words of type k, so a word costs an and, a popc and an add, and each type
// one multiply by its weight.
__device__ __forceinline__ int integrate_typed(const uint32_t *sp, const uint32_t *xr, int N, const uint8_t *tb, int K,
                                               const uint32_t (&wr)[4], uint32_t &syn) {
    int dv = 0;
    for (int k = 0; k < K; ++k) {
        int cnt = 0;
        for (int w = tb[k]; w < tb[k + 1]; ++w) {
            const uint32_t sw = sp[w];
            if (sw == 0u) continue;  // uniform across the core's threads
            cnt += __popc(sw & xr[(size_t)w * N]);
        }
        syn += (uint32_t)cnt;
        dv += weight_of(wr, k) * cnt;
    }
    return dv;
}

__global__ void __launch_bounds__(1024) plain_tick_kernel(const PlainArgs a) {
    extern __shared__ __align__(128) uint32_t xs[];  // [SW][N] crossbar of this core (sorted axons), word-major
    __shared__ uint32_t s[kMaxWords];                 // active axons of this tick (original order)
    __shared__ uint32_t sp[kMaxSortedWords];          // the same, type-sorted order
    __shared__ uint16_t perm[kMaxSortedWords * 32];   // axon at each sorted position
    __shared__ int8_t wt[kMaxSortedWords];            // type of each sorted word
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t red[4];

    const int c = blockIdx.x, b = blockIdx.y, n = threadIdx.x;
    const int AW = a.AW, SW = a.SW, N = a.N;
    const int lane = n & 31, warp = n >> 5;
    const uint32_t xbytes = (uint32_t)N * SW * 4u;

    const size_t bc = (size_t)b * a.C + c;
    uint32_t *row = a.ring + (bc * kRows + (a.tick & (kRows - 1))) * AW;
    if (n < AW) {
        s[n] = row[n];
        row[n] = 0u;
    }
    if (n == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (n < 4) red[n] = 0u;
    __syncthreads();

    // Input lines of this tick (reading: input delay 0).
    if (b < a.n_valid && a.tick < a.in_ticks) {
        const uint32_t *in = a.inputs + ((size_t)b * a.in_ticks + a.tick) * a.in_words;
        for (int k = a.in_ptr[c] + n; k < a.in_ptr[c + 1]; k += blockDim.x) {
            const int L = a.in_line[k];
            if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputLine, L, a.in_words * 32) && ((in[L >> 5] >> (L & 31)) & 1u)) {
                const int ax = a.in_axon[k];
                if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputAxon, ax, a.A)) atomicOr(&s[ax >> 5], 1u << (ax & 31));
            }
        }
    }
    // A core with no active axon this tick needs neither its crossbar nor its
    // weights (dV = 0): with many idle cores the tick is bound by these loads.
    __syncthreads();  // the input bits are in s
    const bool active = __syncthreads_or(n < AW && s[n] != 0u);
    if (active && n == 0) {
        mbar_arrive_expect_tx(&bar, xbytes);
        bulk_g2s(xs, a.xbarT + (size_t)c * N * SW, xbytes, &bar);
    }
    if (active) {
        for (int i = n; i < SW * 32; i += blockDim.x) perm[i] = a.axperm[(size_t)c * SW * 32 + i];
        if (n < SW) wt[n] = a.wtype[(size_t)c * SW + n];
    }
    bool ok = !active || mbar_wait_bounded(&bar, 0);
    if (a.stall_test && blockIdx.x == 0 && blockIdx.y == 0) {
        // Failure-detection test: a barrier that never completes; the bounded
        // wait must give up and report, not hang.
        __shared__ __align__(8) uint64_t never;
        if (n == 0) {
            mbar_init(&never, 1);
            fence_mbar_init();
        }
        __syncthreads();
        ok = ok && mbar_wait_bounded(&never, 0);
    }
    if (__syncthreads_or(!ok)) {
        if (n == 0) atomicExch(a.err, kErrTimeout);
        if (active) mbar_wait_bounded(&bar, 0);  // let the copy land before the CTA exits
        return;
    }

    // Crossbar integration over the type-sorted active axons (word w of
    // neuron n's row at xs[w * N + n]: a warp reads consecutive words, free of
    // bank conflicts); the per-type counts sum to the synaptic events.
    uint32_t syn = 0u;
    int dv = 0;
    if (active) {
        gather_sorted(s, perm, AW, SW, 1, sp, n, blockDim.x);
        __syncthreads();
        const int4 wv = reinterpret_cast<const int4 *>(a.wnk)[(size_t)c * N + n];
        const uint32_t wr[4] = {(uint32_t)wv.x, (uint32_t)wv.y, (uint32_t)wv.z, (uint32_t)wv.w};
        dv = integrate_sorted(sp, xs + n, N, wt, SW, wr, syn);
    }

    // Leak, thresholds, reset.
    const int4 pr = a.prm[(size_t)c * N + n];  // leak, pos_thr, neg_thr, reset
    int *vp = a.V + bc * N + n;
    int v = *vp + dv + pr.x;
    const bool fire = v >= pr.y;
    if (fire)
        v = pr.w;
    else if (v < pr.z)
        v = a.neg_mode ? pr.w : pr.z;
    *vp = v;

    // Spike compaction and delivery.
    const unsigned fm = __ballot_sync(0xffffffffu, fire);
    if (lane == 0) a.spk[bc * a.NW + warp] = fm;
    uint32_t kind = 0u;
    if (fire) {
        const uint2 d = a.dst[(size_t)c * N + n];
        kind = dest_kind(d);
        if (kind == RANC_DEST_CORE) {
            const uint32_t ax = dest_axon(d);
            const long long r = (a.tick + dest_delay(d)) & (kRows - 1);
            if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestCore, d.x, a.C) && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestAxon, ax, a.A))
                atomicOr(a.ring + (((size_t)b * a.C + d.x) * kRows + r) * AW + (ax >> 5), 1u << (ax & 31));
        } else if (kind == RANC_DEST_OUTPUT && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteOutputId, d.x, a.n_out)) {
            atomicAdd(a.out + (size_t)b * a.n_out + d.x, 1u);
            if (a.olog) atomicAdd(a.olog + (size_t)b * a.olog_stride + d.x, 1u);
        }
    }
    const unsigned pm = __ballot_sync(0xffffffffu, kind == RANC_DEST_CORE);
    const unsigned om = __ballot_sync(0xffffffffu, kind == RANC_DEST_OUTPUT);
    const unsigned sy = __reduce_add_sync(0xffffffffu, syn);
    if (lane == 0) {
        atomicAdd(&red[0], (uint32_t)__popc(fm));
        atomicAdd(&red[1], (uint32_t)__popc(pm));
        atomicAdd(&red[2], (uint32_t)__popc(om));
        atomicAdd(&red[3], sy);
    }
    __syncthreads();
    if (n < 4 && b < a.n_valid) a.cnt[bc * 4 + n] += red[n];
}

cudaError_t launch_plain_tick(const PlainArgs &a, cudaStream_t s) {
    const size_t smem = (size_t)a.N * a.SW * 4;
    plain_tick_kernel<<<dim3(a.C, a.B), a.N, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent form of the plain path for ranc_run_samples: one cooperative
// launch runs every sample window.  A CTA owns G cores of one batch slot (one
// thread per neuron, G*N threads), keeps their crossbars in shared memory and
// each neuron's potential, parameters and weights in registers for the whole
// launch; ticks are separated by a grid barrier (bounded wait).  The tick body
// is the one of plain_tick_kernel.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier over all CTAs of a cooperative launch: bar[0] counts
// arrivals without ever being reset (barrier k completes when it reaches
// k * nblocks).  Thread 0 of each CTA arrives with one acquire-release atomic
// (after the CTA barrier, so it publishes the whole CTA's writes) and, unless
// it was the last to arrive, polls with acquire loads.  Returns false if the
// wait gave up.  skip_arrival (failure-detection tests only): this CTA waits
// without arriving, so the barrier cannot complete and every CTA's wait runs
// out.
__device__ bool grid_sync(unsigned *bar, unsigned nblocks, unsigned &gen, int *s_ok, bool skip_arrival = false) {
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        const unsigned target = (gen + 1u) * nblocks;
        unsigned v = 0u;
        if (!skip_arrival)
            asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(v) : "l"(bar) : "memory");
        if (skip_arrival || (v + 1u != target && (int)(ld_acquire_u32(bar) - target) < 0)) {
            const unsigned long long t0 = global_ns();
            while ((int)(ld_acquire_u32(bar) - target) < 0) {
                if (global_ns() - t0 > kWaitLimitNs) {
                    ok = false;
                    break;
                }
            }
        }
        *s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    ++gen;
    return *s_ok != 0;
}

__global__ void __launch_bounds__(1024, 1) plain_window_kernel(const WindowArgs w) {
    extern __shared__ __align__(128) uint32_t sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t red[kMaxWindowCores][4];
    __shared__ int s_ok;
    __shared__ uint8_t tbs[kMaxWindowCores][kMaxTypes + 1];  // sorted words of each type: tbs[kc][k] .. tbs[kc][k+1]
    const PlainArgs &a = w.p;
    const int G = w.G, N = a.N, AW = a.AW, SW = a.SW, C = a.C;
    const int grp = blockIdx.x % w.n_groups, b = blockIdx.x / w.n_groups;
    const int tid = threadIdx.x, cg = tid / N, n = tid % N, lane = tid & 31;
    const int c_first = grp * G, ncores = min(G, C - c_first);
    const int c = c_first + cg;
    const bool has_core = cg < ncores;
    uint32_t *xs = sm;                         // [ncores][SW][N] (word-major, type-sorted axons)
    uint32_t *sb = xs + (size_t)G * N * SW;    // [ncores][AW] active axons of this tick (original order)
    uint32_t *spb = sb + (size_t)G * AW;       // [ncores][SW] the same in sorted order
    uint16_t *perm = reinterpret_cast<uint16_t *>(spb + (size_t)G * SW);  // [ncores][SW*32] axon at each sorted position
    int8_t *wt = reinterpret_cast<int8_t *>(perm + (size_t)G * SW * 32);  // [ncores][SW] type of each sorted word
    uint32_t *inb = reinterpret_cast<uint32_t *>(wt + (((size_t)G * SW + 15) & ~(size_t)15));  // [t_in][in_words] inputs
    // With w.in_cap, the group's input-line entries: line, and (core in the group, axon) as one bit position of sb.
    uint32_t *lns = inb + (w.stream ? 0 : (size_t)w.t_in * a.in_words);  // [in_cap]
    uint16_t *lpos = reinterpret_cast<uint16_t *>(lns + w.in_cap);       // [in_cap]
    const unsigned nblocks = gridDim.x;
    unsigned gen = 0;

    const uint32_t xbytes = (uint32_t)ncores * N * SW * 4u;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, xbytes);
        bulk_g2s(xs, a.xbarT + (size_t)c_first * N * SW, xbytes, &bar);
    }
    for (int i = tid; i < ncores * SW * 32; i += blockDim.x) perm[i] = a.axperm[(size_t)c_first * SW * 32 + i];
    for (int i = tid; i < ncores * SW; i += blockDim.x) wt[i] = a.wtype[(size_t)c_first * SW + i];
    int lam = 0, pth = 0, nth = 0, rst = 0, v0 = 0;
    uint32_t wr[4] = {0u, 0u, 0u, 0u};
    uint2 dd = make_uint2(0u, 0u);
    if (has_core) {
        const int4 pr = a.prm[(size_t)c * N + n];
        lam = pr.x;
        pth = pr.y;
        nth = pr.z;
        rst = pr.w;
        const int4 wv = reinterpret_cast<const int4 *>(a.wnk)[(size_t)c * N + n];
        wr[0] = (uint32_t)wv.x;
        wr[1] = (uint32_t)wv.y;
        wr[2] = (uint32_t)wv.z;
        wr[3] = (uint32_t)wv.w;
        dd = a.dst[(size_t)c * N + n];
        v0 = w.v0[(size_t)c * N + n];
    }
    if (tid < kMaxWindowCores * 4) red[tid / 4][tid % 4] = 0u;
    __syncthreads();
    const bool ok0 = mbar_wait_bounded(&bar, 0);
    if (__syncthreads_or(!ok0)) {
        if (tid == 0) atomicExch(a.err, kErrTimeout);
        mbar_wait_bounded(&bar, 0);
        return;
    }
    for (int i = tid; i < ncores * (a.K + 1); i += blockDim.x) {  // ordered before use by the first grid barrier
        const int kc = i / (a.K + 1), k = i % (a.K + 1);
        int nw = 0;
        for (int q = 0; q < SW; ++q) {
            const int ty = wt[kc * SW + q];
            nw += (ty >= 0 && ty < k) ? 1 : 0;
        }
        tbs[kc][k] = (uint8_t)nw;
    }
    // Gather into the sorted order: the (word, bit) of sb read for each of
    // this thread's sorted positions is the same every tick; up to two
    // positions per thread are kept in registers (0xFFFFFFFF: no axon).
    const int gP = ncores * SW * 32;
    const bool g_regs = gP <= 2 * (int)blockDim.x;
    uint32_t gsrc[2] = {0xFFFFFFFFu, 0xFFFFFFFFu};
    if (g_regs)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = tid + q * (int)blockDim.x;
            if (i < gP) {
                const int j = i / (SW * 32), ia = perm[i];
                if (ia != 0xFFFF) gsrc[q] = ((uint32_t)(j * AW + (ia >> 5)) << 5) | (uint32_t)(ia & 31);
            }
        }
    const uint32_t kind = dest_kind(dd);
    const int ipw = w.t_in * a.in_words;
    const int ip0 = a.in_ptr[c_first], ip1 = a.in_ptr[c_first + ncores];
    if (w.in_cap)  // read once per launch instead of every input tick (the first grid barrier orders it)
        for (int k = ip0 + tid; k < ip1; k += blockDim.x) {
            int kc = 0;
            while (kc + 1 < ncores && k >= a.in_ptr[c_first + kc + 1]) ++kc;
            lns[k - ip0] = (uint32_t)a.in_line[k];
            lpos[k - ip0] = (uint16_t)(kc * AW * 32 + a.in_axon[k]);
        }
    uint32_t n_sp = 0, n_pk = 0, n_ou = 0, n_syn = 0;
    uint32_t oc = 0u;  // this neuron's output-bus events in the current window
    int V = v0;
    const int n_windows = (w.n_samples + a.B - 1) / a.B;
    for (int win = 0; win < n_windows; ++win) {
        const int smp = win * a.B + b;
        const bool valid = smp < w.n_samples;
        // Window start (every sample starts from V = v0 and empty rows): V = v0, this CTA's scheduler rows and
        // (group 0) output row cleared.
        V = v0;
        uint32_t *rows = a.ring + ((size_t)b * C + c_first) * kRows * AW;
        for (int i = tid; i < ncores * kRows * AW; i += blockDim.x) __stcg(rows + i, 0u);
        if (grp == 0)
            for (int i = tid; i < a.n_out; i += blockDim.x) __stcg(a.out + (size_t)b * a.n_out + i, 0u);
        if (!w.stream)
            for (int i = tid; i < ipw; i += blockDim.x) inb[i] = valid ? __ldg(a.inputs + (size_t)smp * ipw + i) : 0u;
        // Failure-detection test: CTA 0 does not arrive at the first barrier.
        if (!grid_sync(w.bar, nblocks, gen, &s_ok, a.stall_test && blockIdx.x == 0 && win == 0)) break;
        bool stop = false;
        for (int t = 0; t < w.window; ++t) {
            const int r = t & (kRows - 1);
            for (int i = tid; i < ncores * AW; i += blockDim.x) {
                uint32_t *p = a.ring + (((size_t)b * C + c_first + i / AW) * kRows + r) * AW + i % AW;
                sb[i] = __ldcg(p);
                __stcg(p, 0u);
            }
            __syncthreads();
            if (valid && t < w.t_in) {
                // Inputs of tick t: staged in shared memory, or (streaming) read
                // from the caller's array, one frame per tick.
                const uint32_t *in = w.stream ? a.inputs + ((size_t)smp * w.t_in + t) * a.in_words
                                              : inb + (size_t)t * a.in_words;
                if (w.in_cap)
                    for (int e = tid; e < ip1 - ip0; e += blockDim.x) {
                        const uint32_t L = lns[e];
                        if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputLine, L, a.in_words * 32) && ((in[L >> 5] >> (L & 31)) & 1u)) {
                            const uint32_t p = lpos[e];
                            if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputAxon, p, ncores * AW * 32)) atomicOr(&sb[p >> 5], 1u << (p & 31));
                        }
                    }
                else
                for (int k = ip0 + tid; k < ip1; k += blockDim.x) {
                    const int L = a.in_line[k];
                    if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputLine, L, a.in_words * 32) && ((in[L >> 5] >> (L & 31)) & 1u)) {
                        int kc = 0;
                        while (kc + 1 < ncores && k >= a.in_ptr[c_first + kc + 1]) ++kc;
                        const int ax = a.in_axon[k];
                        if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputAxon, ax, a.A)) atomicOr(&sb[kc * AW + (ax >> 5)], 1u << (ax & 31));
                    }
                }
                __syncthreads();
            }
            if (g_regs) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int i = tid + q * (int)blockDim.x;
                    if (i >= ((gP + 31) & ~31)) break;  // uniform per warp
                    const uint32_t g = gsrc[q];
                    const bool on = g != 0xFFFFFFFFu && ((sb[g >> 5] >> (g & 31)) & 1u);
                    const unsigned word = __ballot_sync(0xffffffffu, on);
                    if ((i & 31) == 0) spb[i >> 5] = word;
                }
            } else {
                gather_sorted(sb, perm, AW, SW, ncores, spb, tid, blockDim.x);
            }
            __syncthreads();
            bool fire = false;
            if (has_core) {
                uint32_t syn = 0u;
                const int dv = integrate_typed(spb + cg * SW, xs + (size_t)cg * SW * N + n, N, tbs[cg], a.K, wr, syn);
                int x = V + dv + lam;
                fire = x >= pth;
                if (fire)
                    x = rst;
                else if (x < nth)
                    x = a.neg_mode ? rst : nth;
                V = x;
                if (valid) {
                    n_syn += syn;
                    n_sp += fire ? 1u : 0u;
                }
                if (fire) {
                    if (kind == RANC_DEST_CORE) {
                        const uint32_t ax = dest_axon(dd);
                        const int rr = (t + (int)dest_delay(dd)) & (kRows - 1);
                        if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestCore, dd.x, C) && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestAxon, ax, a.A))
                            atomicOr(a.ring + (((size_t)b * C + dd.x) * kRows + rr) * AW + (ax >> 5), 1u << (ax & 31));
                        if (valid) ++n_pk;
                    } else if (kind == RANC_DEST_OUTPUT) {
                        ++oc;  // added to the output bus once, at the window's last tick
                        if (valid) {
                            ++n_ou;
                            if (w.olog && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteOutputId, dd.x, a.n_out))
                                atomicAdd(w.olog + ((size_t)smp * w.window + t) * a.n_out + dd.x, 1u);
                        }
                    }
                }
            }
            if (t == w.window - 1 && oc) {
                if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteOutputId, dd.x, a.n_out)) atomicAdd(a.out + (size_t)b * a.n_out + dd.x, oc);
                oc = 0u;
            }
            const unsigned fm = __ballot_sync(0xffffffffu, fire);
            if (has_core && lane == 0) a.spk[((size_t)b * C + c) * a.NW + n / 32] = fm;
            if (!grid_sync(w.bar, nblocks, gen, &s_ok)) {
                stop = true;
                break;
            }
        }
        if (stop) break;
        if (grp == 0 && valid && w.counts)
            for (int i = tid; i < a.n_out; i += blockDim.x)
                w.counts[(size_t)smp * a.n_out + i] = __ldcg(a.out + (size_t)b * a.n_out + i);
        if (!grid_sync(w.bar, nblocks, gen, &s_ok)) break;
    }
    if (!s_ok) {
        if (tid == 0) atomicExch(a.err, kErrTimeout);
        return;
    }
    if (has_core) a.V[((size_t)b * C + c) * N + n] = V;
    // Counters: per core of this CTA, summed over its valid windows.
    n_sp = __reduce_add_sync(0xffffffffu, n_sp);
    n_pk = __reduce_add_sync(0xffffffffu, n_pk);
    n_ou = __reduce_add_sync(0xffffffffu, n_ou);
    n_syn = __reduce_add_sync(0xffffffffu, n_syn);
    if (has_core && lane == 0) {
        atomicAdd(&red[cg][0], n_sp);
        atomicAdd(&red[cg][1], n_pk);
        atomicAdd(&red[cg][2], n_ou);
        atomicAdd(&red[cg][3], n_syn);
    }
    __syncthreads();
    if (tid < ncores * 4) a.cnt[((size_t)b * C + c_first + tid / 4) * 4 + tid % 4] += red[tid / 4][tid % 4];
}

// Launches plain_window_kernel when its grid fits on the device at once (the
// barrier needs every CTA resident); returns cudaErrorCooperativeLaunchTooLarge
// otherwise, so the caller can use the per-tick launches instead.
cudaError_t launch_plain_windows(const WindowArgs &w_in, cudaStream_t s) {
    WindowArgs w = w_in;
    const int threads = w.G * w.p.N;
    const size_t base = ((size_t)w.G * w.p.N * w.p.SW + (size_t)w.G * w.p.AW + (size_t)w.G * w.p.SW) * 4 +
                        (size_t)w.G * w.p.SW * 32 * 2 + (((size_t)w.G * w.p.SW + 15) & ~(size_t)15) +
                        (w.stream ? 0 : (size_t)w.t_in * w.p.in_words) * 4;
    // The input-line entries go to shared memory when they fit (6 bytes each).
    if (w.in_cap > 0 && base + (size_t)w.in_cap * 6 + 64 > 200 * 1024) w.in_cap = 0;
    const size_t smem = base + (w.in_cap > 0 ? (size_t)w.in_cap * 6 + 16 : 0);
    cudaError_t e = raise_smem_limit((const void *)plain_window_kernel, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plain_window_kernel, threads, smem)) != cudaSuccess)
        return e;
    const int grid = w.n_groups * w.p.B;
    if ((long long)per_sm * n_sm < grid) return cudaErrorCooperativeLaunchTooLarge;
    if ((e = cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
    void *args[] = {&w};
    return cudaLaunchCooperativeKernel((const void *)plain_window_kernel, dim3(grid), dim3(threads), args, smem, s);
}

// ---------------------------------------------------------------------------
// Persistent form of ranc_step on the plain path: n ticks in one cooperative
// launch, for grids of any size.  Work units are (sample, core) pairs, dealt
// to the CTAs in turn (the same ones every tick); ticks are separated by the
// grid barrier.  A CTA (1024 threads) runs each tick in phases over all its
// units at once, so that the loads of many units are in flight together:
//   A  scheduler rows read and cleared, input lines ORed in, activity flags;
//   B  crossbar integration of the active units, one at a time (crossbar
//      words read from global memory / L2, type-sorted as in plain_tick_kernel);
//   C  leak, thresholds and reset of every neuron of every unit, four at a
//      time per thread with their loads issued first; spike words, delivery,
//      output bus, counters.
// ---------------------------------------------------------------------------

constexpr int kMaxStepUnits = 64;  // units per CTA and tick held in shared memory

__global__ void __launch_bounds__(1024, 1) plain_steps_kernel(const PlainArgs a, int n_ticks, unsigned *bar, int resident) {
    extern __shared__ __align__(16) uint32_t smp[];
    __shared__ uint32_t red[kMaxStepUnits][4];
    __shared__ int act_sh[kMaxStepUnits];
    __shared__ int ub_sh[kMaxStepUnits], uc_sh[kMaxStepUnits];  // sample and core of each unit
    __shared__ long long uv_sh[kMaxStepUnits];  // (b * C + c) * N: the unit's first potential
    __shared__ long long us_sh[kMaxStepUnits];  // (b * C + c) * NW: the unit's first spike word
    __shared__ int up_sh[kMaxStepUnits];        // c * N: the unit's first parameter
    __shared__ int s_ok;
    const int N = a.N, AW = a.AW, SW = a.SW, C = a.C;
    const int tid = threadIdx.x, lane = tid & 31, nt = blockDim.x;
    const int n_units = C * a.B;
    const int m = (n_units - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // units of this CTA
    int *dvs = reinterpret_cast<int *>(smp);                        // [m][N] dV of the active units
    uint32_t *sb = reinterpret_cast<uint32_t *>(dvs + (size_t)m * N);  // [m][AW] active axons
    uint32_t *spb = sb + m * AW;                                    // [SW] sorted active axons of one unit
    uint16_t *perm = reinterpret_cast<uint16_t *>(spb + SW);        // [SW * 32]
    int8_t *wt = reinterpret_cast<int8_t *>(perm + SW * 32);        // [SW]
    // With `resident`, the potentials and parameters of the CTA's units stay in
    // shared memory for the whole launch (the units are the same every tick):
    // loaded here, written back after the last tick.
    int4 *prs = reinterpret_cast<int4 *>(smp + (((size_t)m * N + (size_t)m * AW + SW + (SW * 32 + 1) / 2 + (SW + 3) / 4 + 3) & ~(size_t)3));
    int *vs = reinterpret_cast<int *>(prs + (size_t)m * N);         // [m][N]
    auto unit = [&](int i) { return (int)blockIdx.x + i * (int)gridDim.x; };  // b * C + c
    unsigned gen = 0;
    if (tid == 0) s_ok = 1;
    for (int i = tid; i < m; i += nt) {
        ub_sh[i] = unit(i) / C;
        uc_sh[i] = unit(i) % C;
        uv_sh[i] = (long long)unit(i) * N;
        us_sh[i] = (long long)unit(i) * a.NW;
        up_sh[i] = unit(i) % C * N;
    }
    // Phase C: thread tid updates neuron tid % N of units (round * upr + tid / N).
    const int upr = nt / N, my_slot = tid / N, my_n = tid % N;
    __syncthreads();
    if (resident)
        for (int i = tid; i < m * N; i += nt) {
            const int k = i / N, n = i - k * N;
            vs[i] = a.V[uv_sh[k] + n];
            prs[i] = a.prm[up_sh[k] + n];
        }
    // Per-tick counters and activity flags start at zero (each tick zeroes
    // them again after use, before the grid barrier that ends it).
    for (int i = tid; i < m * 4; i += nt) red[i / 4][i % 4] = 0u;
    for (int i = tid; i < m; i += nt) act_sh[i] = 0;
    __syncthreads();
    for (int t = 0; t < n_ticks; ++t) {
        const long long tick = a.tick + t;
        const int r0 = (int)(tick & (kRows - 1));
        // ---- A: rows, inputs, activity
        for (int i = tid; i < m * AW; i += nt) {
            const int k = i / AW;
            uint32_t *row = a.ring + (((size_t)ub_sh[k] * C + uc_sh[k]) * kRows + r0) * AW + (i - k * AW);
            const uint32_t w = *row;
            sb[i] = w;
            if (w) {
                *row = 0u;
                act_sh[k] = 1;
            }
        }
        __syncthreads();
        if (tick < a.in_ticks) {
            for (int i = 0; i < m; ++i) {
                const int b = ub_sh[i], c = uc_sh[i];
                if (b >= a.n_valid) continue;
                const uint32_t *in = a.inputs + ((size_t)b * a.in_ticks + tick) * a.in_words;
                for (int k = a.in_ptr[c] + tid; k < a.in_ptr[c + 1]; k += nt) {
                    const int L = a.in_line[k];
                    if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputLine, L, a.in_words * 32) && ((in[L >> 5] >> (L & 31)) & 1u)) {
                        const int ax = a.in_axon[k];
                        if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteInputAxon, ax, a.A)) atomicOr(&sb[i * AW + (ax >> 5)], 1u << (ax & 31));
                        act_sh[i] = 1;
                    }
                }
            }
            __syncthreads();
        }
        // ---- B: integration of the active units
        for (int i = 0; i < m; ++i) {
            if (!act_sh[i]) continue;  // uniform over the CTA
            const int c = uc_sh[i];
            for (int k = tid; k < SW * 32; k += nt) perm[k] = a.axperm[(size_t)c * SW * 32 + k];
            for (int k = tid; k < SW; k += nt) wt[k] = a.wtype[(size_t)c * SW + k];
            __syncthreads();
            if (tid < ((SW * 32 + 31) & ~31)) gather_sorted(sb + i * AW, perm, AW, SW, 1, spb, tid, nt);
            __syncthreads();
            for (int n = tid; n < N; n += nt) {
                const int4 wv = reinterpret_cast<const int4 *>(a.wnk)[(size_t)c * N + n];
                const uint32_t wr[4] = {(uint32_t)wv.x, (uint32_t)wv.y, (uint32_t)wv.z, (uint32_t)wv.w};
                uint32_t syn = 0u;
                dvs[i * N + n] = integrate_sorted(spb, a.xbarT + (size_t)c * SW * N + n, N, wt, SW, wr, syn);
                syn = __reduce_add_sync(0xffffffffu, syn);
                if (lane == 0 && syn) atomicAdd(&red[i][3], syn);
            }
            __syncthreads();
        }
        // ---- C: neuron updates of every unit: four units per thread per round,
        // their loads issued first
        for (int i0 = 0; i0 < m; i0 += 4 * upr) {
            int vv[4];
            int4 pr[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * upr + my_slot;
                if (my_slot >= upr || i >= m) break;  // uniform per warp (N is a multiple of 32)
                vv[q] = resident ? vs[i * N + my_n] : a.V[uv_sh[i] + my_n];
                pr[q] = resident ? prs[i * N + my_n] : a.prm[up_sh[i] + my_n];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * upr + my_slot;
                if (my_slot >= upr || i >= m) break;
                const int n = my_n;
                const long long vo = uv_sh[i];
                int v = vv[q] + (act_sh[i] ? dvs[i * N + n] : 0) + pr[q].x;
                const bool fire = v >= pr[q].y;
                if (fire)
                    v = pr[q].w;
                else if (v < pr[q].z)
                    v = a.neg_mode ? pr[q].w : pr[q].z;
                if (resident) vs[i * N + n] = v;
                else a.V[vo + n] = v;
                const unsigned fm = __ballot_sync(0xffffffffu, fire);
                if (lane == 0) a.spk[us_sh[i] + n / 32] = fm;
                uint32_t kind = 0u;
                if (fire) {
                    const int b = ub_sh[i];
                    const uint2 d = a.dst[(size_t)up_sh[i] + n];
                    kind = dest_kind(d);
                    if (kind == RANC_DEST_CORE) {
                        const uint32_t ax = dest_axon(d);
                        const long long r = (tick + dest_delay(d)) & (kRows - 1);
                        if (RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestCore, d.x, C) && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteDestAxon, ax, a.A))
                            atomicOr(a.ring + (((size_t)b * C + d.x) * kRows + r) * AW + (ax >> 5), 1u << (ax & 31));
                    } else if (kind == RANC_DEST_OUTPUT && RANC_IN_RANGE(a.err, a.dbg_plant, kSiteOutputId, d.x, a.n_out)) {
                        atomicAdd(a.out + (size_t)b * a.n_out + d.x, 1u);
                    }
                }
                if (fm) {
                    const unsigned pm = __ballot_sync(0xffffffffu, kind == RANC_DEST_CORE);
                    const unsigned om = __ballot_sync(0xffffffffu, kind == RANC_DEST_OUTPUT);
                    if (lane == 0) {
                        atomicAdd(&red[i][0], (uint32_t)__popc(fm));
                        if (pm) atomicAdd(&red[i][1], (uint32_t)__popc(pm));
                        if (om) atomicAdd(&red[i][2], (uint32_t)__popc(om));
                    }
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < m * 4; i += nt) {  // each thread zeroes what it read
            const int k = i >> 2;
            if (ub_sh[k] < a.n_valid && red[k][i & 3])
                a.cnt[((size_t)ub_sh[k] * C + uc_sh[k]) * 4 + (i & 3)] += red[k][i & 3];
            red[k][i & 3] = 0u;
        }
        for (int i = tid; i < m; i += nt) act_sh[i] = 0;  // read by phase C, before the barrier above
        // Failure-detection test: CTA 0 does not arrive at the first barrier.
        if (!grid_sync(bar, gridDim.x, gen, &s_ok, a.stall_test && blockIdx.x == 0 && t == 0)) {
            if (tid == 0) atomicExch(a.err, kErrTimeout);
            return;
        }
    }
    if (resident)  // every update is in shared memory: the last grid barrier synchronised the CTA
        for (int i = tid; i < m * N; i += nt) {
            const int k = i / N;
            a.V[uv_sh[k] + (i - k * N)] = vs[i];
        }
}

size_t plain_steps_smem(int m, int N, int AW, int SW, bool resident) {
    const size_t words = ((size_t)m * N + (size_t)m * AW + SW + (SW * 32 + 1) / 2 + (SW + 3) / 4 + 3) & ~(size_t)3;
    return words * 4 + (resident ? (size_t)m * N * 20 : 16);
}

// n_ticks ticks of the plain path in one cooperative launch; the grid is the
// number of CTAs that fit on the device at once, and at least as many as
// needed for kMaxStepUnits units per CTA (otherwise cudaErrorCooperativeLaunchTooLarge).
cudaError_t launch_plain_steps(const PlainArgs &a, int n_ticks, unsigned *bar, cudaStream_t s) {
    const int threads = 1024;
    const long long units = (long long)a.C * a.B;
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const long long grid = std::min<long long>(units, n_sm);  // one CTA per SM
    const int m = (int)((units + grid - 1) / grid);
    if (m > kMaxStepUnits) return cudaErrorCooperativeLaunchTooLarge;
    // Potentials and parameters resident in shared memory when they fit.
    int resident = plain_steps_smem(m, a.N, a.AW, a.SW, true) <= 200 * 1024 ? 1 : 0;
    const size_t smem = plain_steps_smem(m, a.N, a.AW, a.SW, resident != 0);
    if (smem > 200 * 1024) return cudaErrorCooperativeLaunchTooLarge;  // per-tick launches instead
    if ((e = raise_smem_limit((const void *)plain_steps_kernel, (int)smem)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plain_steps_kernel, threads, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    if ((e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
    PlainArgs args = a;
    void *params[] = {&args, &n_ticks, &bar, &resident};
    return cudaLaunchCooperativeKernel((const void *)plain_steps_kernel, dim3((unsigned)grid), dim3(threads), params, smem, s);
}

// V <- v0 for every sample.
__global__ void plain_reset_v_kernel(int *V, const int *v0, long long per_sample, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        V[i] = v0[i % per_sample];
}

cudaError_t plain_setup_kernel_attrs(int N, int SW) {
    const int smem = N * SW * 4;
    if (smem <= 48 * 1024) return cudaSuccess;
    return raise_smem_limit((const void *)plain_tick_kernel, smem);
}

// Raises (never lowers) a kernel's dynamic shared-memory limit: the attribute
// is shared by every handle of the process.
cudaError_t raise_smem_limit(const void *kernel, int bytes) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_plain_reset(ranc_sim *sim, bool counters) {
    const long long per = (long long)sim->C * sim->N, total = per * sim->B;
    cudaError_t e;
    plain_reset_v_kernel<<<(unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096), 256, 0,
                           sim->stream>>>((int *)sim->V, sim->v0, per, total);
    sim->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t ring_bytes = (size_t)sim->B * sim->C * kRows * (sim->A / 32) * 4;
    if ((e = cudaMemsetAsync(sim->ring, 0, ring_bytes, sim->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sim->spk, 0, (size_t)sim->B * sim->C * (sim->N / 32) * 4, sim->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(sim->out, 0, (size_t)sim->B * sim->n_outputs * 4, sim->stream)) != cudaSuccess)
        return e;
    if (counters && (e = cudaMemsetAsync(sim->cnt, 0, sim->cnt_len * 8, sim->stream)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Order-independent state digest: sum of splitmix64_mix((i << 32) | (uint32)V[i]).
__global__ void digest_kernel(const int *V, long long n, unsigned long long *out) {
    unsigned long long acc = 0ull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += splitmix64_mix(((unsigned long long)i << 32) | (uint32_t)V[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

cudaError_t launch_digest(const int *V, long long n, unsigned long long *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, 8, s);
    if (e != cudaSuccess) return e;
    long long blocks = (n + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    if (blocks < 1) blocks = 1;
    digest_kernel<<<(unsigned)blocks, 256, 0, s>>>(V, n, out);
    return cudaGetLastError();
}

}  // namespace ranc
