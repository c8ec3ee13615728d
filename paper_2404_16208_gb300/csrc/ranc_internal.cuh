// Internal declarations of the RANC CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ranc.h"

namespace ranc {

constexpr int kRows = RANC_ROWS;     // scheduler rows (Sec. III-E); delays 1..15
constexpr int kMaxTypes = 8;         // weight slots per neuron
constexpr int kMaxWords = 32;        // axons/32 and neurons/32 upper bound (1024)
constexpr int kMaxSortedWords = kMaxWords + kMaxTypes;  // words of the type-sorted axon order (each type word-aligned)
constexpr int kTileS = 128;          // samples per tensor-core tile (batched path)
// Storage of the batched path's potentials (values of RANC_POTENTIAL_*).
constexpr int kVInt32 = 0, kVInt16 = 1, kVHalf = 2;
constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;  // static scratch of the allocation-free read

// Device error word values (set by kernels, read by synchronous host calls).
// kErrBounds carries the site of the failed check in bits 8 and up.
enum : int { kErrNone = 0, kErrTimeout = 1, kErrBounds = 2 };

// Debug builds (compiled with -DRANC_DEBUG, library libranc_debug.so): every
// index a kernel derives from the network description before a global access
// is checked against its range -- the input line of a fan-in entry, the axon
// of an input entry, the destination core and axon of a spike packet, the
// output id of an output-bus event.  A failed check skips that access and
// records kErrBounds | site << 8 in the handle's error word (the first failure
// is kept); the synchronous call that reads the word returns RANC_ECUDA naming
// the site.  `plant` (from the RANC_DEBUG_PLANT environment variable at
// create, debug builds only) fails every check of one site on purpose, so
// that tests can see a failure reported without any invalid access.  Release
// builds compile every check to `true`.
enum : int { kSiteInputLine = 1, kSiteInputAxon = 2, kSiteDestCore = 3, kSiteDestAxon = 4, kSiteOutputId = 5 };
#ifdef RANC_DEBUG
constexpr bool kDebugBuild = true;
__device__ __forceinline__ bool debug_in_range(int *err, int plant, int site, long long i, long long n) {
    if (i >= 0 && i < n && site != plant) return true;
    atomicCAS(err, kErrNone, kErrBounds | (site << 8));
    return false;
}
#define RANC_IN_RANGE(err, plant, site, i, n) ::ranc::debug_in_range((err), (plant), (site), (long long)(i), (long long)(n))
#else
constexpr bool kDebugBuild = false;
#define RANC_IN_RANGE(err, plant, site, i, n) true
#endif

// Resolved destination of a neuron: x = destination core (kind core) or output
// id (kind output); y = axon | delay << 16 | kind << 24.
__host__ __device__ inline uint32_t dest_axon(uint2 d) { return d.y & 0xFFFFu; }
__host__ __device__ inline uint32_t dest_delay(uint2 d) { return (d.y >> 16) & 0xFFu; }
__host__ __device__ inline uint32_t dest_kind(uint2 d) { return d.y >> 24; }

// Per-launch parameters of the plain (one thread per neuron) tick kernel.
struct PlainArgs {
    int C, A, N, K, AW, NW, B;   // cores, axons, neurons, types, A/32, N/32, batch
    int SW;                      // words of the type-sorted axon order (same for every core)
    int n_valid;                 // samples b < n_valid receive inputs
    int in_words, in_ticks, n_out, neg_mode;
    long long tick;              // tick being simulated (counted from reset)
    // The plain kernels integrate over the axons of each core sorted by type
    // (then by index), every type starting at a 32-position boundary: position
    // p holds axon axperm[c][p] (0xFFFF: none), and word w holds only type
    // wtype[c][w] (-1: no axon).  Scheduler rows, inputs and packets keep the
    // original axon numbers; a tick gathers its active axons into this order.
    const uint32_t *xbarT;       // [C][SW][N]   crossbar bits in sorted order: word w of neuron n's row at [c][w][n]
    const int8_t *wtype;         // [C][SW]      type of each sorted word
    const uint16_t *axperm;      // [C][SW*32]   axon at each sorted position
    const int16_t *wnk;          // [C][N][8]    weight per (neuron, type)
    const int4 *prm;             // [C][N]       {leak, pos_thr, neg_thr, reset}
    const uint2 *dst;            // [C][N]       resolved destination
    const int *in_ptr;           // [C+1]        per-core list of (input line, axon)
    const int *in_line, *in_axon;
    const uint32_t *inputs;      // [B][in_ticks][in_words]
    int *V;                      // [B][C][N]
    uint32_t *ring;              // [B][C][kRows][AW]
    uint32_t *spk;               // [B][C][NW]   spikes of the last tick
    uint32_t *out;               // [B][n_out]
    unsigned long long *cnt;     // [B][C][4]    spikes, packets, outputs, synaptic events
    int *err;
    int stall_test;              // test only: CTA (0, 0) waits on an mbarrier nothing arrives on (per-tick
                                 // kernel); CTA 0 skips its first grid-barrier arrival (persistent kernel)
    uint32_t *olog;              // NULL, or this tick's output-bus log: event (b, id) also adds 1 at
    long long olog_stride;       //   olog[b * olog_stride + id]
    int dbg_plant;               // debug builds: site whose range checks fail on purpose (0: none)
};

// Persistent plain path (ranc_run_samples): G cores per CTA, all windows in one launch.
constexpr int kMaxWindowCores = 32;
struct WindowArgs {
    PlainArgs p;                 // p.inputs = [n_samples][t_in][in_words]
    int G, n_groups;             // cores per CTA, CTAs per batch slot
    int n_samples, t_in, window;
    const int *v0;               // [C][N]
    uint32_t *counts;            // [n_samples][n_out] (device) or NULL
    unsigned *bar;               // [2] grid barrier: arrivals, generation
    int stream;                  // inputs read from p.inputs every tick instead of staged in shared memory
    int in_cap;                  // > 0: the group's (line, axon) entries staged in shared memory (capacity)
    uint32_t *olog;              // NULL, or per-tick output-bus log [n_samples][window][n_out]
};

// Batched-path device layout (one tile = kTileS samples, sample-minor bits).
struct BatchedArgs {
    int C, A, N, AW, T;          // cores, axons, neurons, A/32, number of sample tiles
    int n_valid;                 // real samples (the rest of the last tile is padding)
    int in_words, in_ticks, n_out, neg_mode;
    long long tick;
    const int4 *prm;             // [C][N]
    const uint2 *dst;            // [C][N]
    const int *in_ptr, *in_line, *in_axon;   // per-core (line, axon) lists
    const uint32_t *inT;         // [T][in_ticks][n_inputs][4] sample-minor input bits
    int n_inputs;
    void *V;                     // [T][C][N/32][kTileS][32] int16 or int32
    uint32_t *ring;              // [T][C][kRows][A][4] sample-minor scheduler rows
    uint32_t *out;               // [B_pad][n_out]
    unsigned long long *cnt;     // [T][C][4]
    int *err;
};

}  // namespace ranc

// Host-side handle.
struct ranc_sim {
    // shape
    int C = 0, A = 0, N = 0, K = 0, B = 0, path = 0, neg_mode = 0;
    int grid_w = 0, grid_h = 0, n_inputs = 0, n_outputs = 0, in_words = 0, weight_bits = 0;
    int B_pad = 0, T = 0, vmode = 0;    // batched path: padded batch, tiles, potential storage (kVInt32 ...)
    int v_lazy = 0;                     // batched: V and spike masks are the reset values, not yet written
    int ring_all_dirty = 1;             // batched: any scheduler row may hold bits (full clear on reset)
    int max_delay = 15;                 // batched: largest core-to-core delay of the network
    uint32_t sclock = 2048;             // batched: stamp clock of the next tick (== tick mod 16)
    int all_active_ticks = 0;           // batched: ticks left in which every item counts as active
    int pend_dirty = 0;                 // batched: some item may hold deferred idle ticks
    cudaStream_t stream = nullptr;
    int device = 0;

    // constant network arrays (device)
    uint32_t *xbarT = nullptr;
    int8_t *wtype = nullptr;            // plain: [C][SW] type of each word of the type-sorted axon order
    uint16_t *axperm = nullptr;         // plain: [C][SW*32] axon at each type-sorted position
    int SW = 0;                         // plain: words of that order
    int in_group_max = 0;               // plain: most input-line entries of one window-kernel core group
    int dbg_plant = 0;                  // debug builds: RANC_DEBUG_PLANT at create (see RANC_IN_RANGE)
    int16_t *wnk = nullptr;
    int4 *prm = nullptr;
    uint2 *dst = nullptr;
    int *in_ptr = nullptr, *in_line = nullptr, *in_axon = nullptr;
    int *v0 = nullptr;
    void *wfold = nullptr;              // batched: [C][N][A] fp16 folded weights
    void *tmap = nullptr;               // batched: path-specific host state (tensor map, tables)
    void *multi = nullptr;              // multi-network handle (ranc_create_multi): its host state
    long long nps = 0;                  // neurons per sample (C * N, or the sum over a multi handle's networks)

    // state (device)
    void *V = nullptr;
    uint32_t *ring = nullptr, *spk = nullptr, *out = nullptr;
    unsigned long long *cnt = nullptr;  // per (sample or tile, core) partial counters
    size_t cnt_len = 0;
    uint32_t *inputs = nullptr;         // plain: [B][ticks][words]; batched: [T][ticks][n_inputs][4]
    size_t inputs_cap = 0;
    int in_ticks = 0;
    const uint32_t *in_override = nullptr;  // plain: caller's device slice used by run_samples
    uint32_t *stage = nullptr;          // batched: staging buffer for untransposed inputs
    size_t stage_cap = 0;
    int *err = nullptr;
    unsigned long long *digest = nullptr;
    unsigned *gbar = nullptr;            // plain: grid barrier of the persistent window kernel
    uint32_t *counts_dev = nullptr;      // plain: device copy of run_samples counts (host mode)
    size_t counts_cap = 0;
    uint32_t *olog_dev = nullptr;        // run_stream: device copy of the per-tick output log (host mode)
    size_t olog_cap = 0;
    uint32_t *olog_t = nullptr;          // run_stream: log slot of the tick being stepped, or NULL
    long long olog_stride = 0;
    int n_valid = 0;

    long long tick = 0;
    unsigned long long ticks_total = 0;  // RANC_CNT_TICKS
    long long launches = 0;

    // kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<long long> ev_ticks;     // ticks advanced by the kernel between each event pair
    int ev_used = 0;
    double timed_ms = 0.0;
    long long timed_launches = 0;

    // run_samples on the batched path with device buffers: the window sequence
    // recorded as a CUDA graph, replayed while its arguments stay the same
    cudaGraphExec_t win_exec = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream the sequence is recorded on
    struct WinKey {
        const void *inputs = nullptr, *counts = nullptr, *inT = nullptr;
        int n_samples = -1, t_in = -1, window = -1;
        bool operator==(const WinKey &o) const {
            return inputs == o.inputs && counts == o.counts && inT == o.inT && n_samples == o.n_samples &&
                   t_in == o.t_in && window == o.window;
        }
    } win_key;
    bool win_timed = false;              // the recording brackets each group's ticks with timing events
    std::vector<cudaEvent_t> win_events; // [groups][2] timing events recorded by the graph (owned)
    int win_pending = 0;                 // replays whose timing events are not folded yet (0 or 1)
    long long win_launches = 0;          // kernels in the recorded sequence
    unsigned long long win_ticks = 0;    // sample ticks it advances
    long long win_tick_after = 0;        // tick counter after it
    uint32_t win_sclock_after = 0;       // batched stamp clock after it
    int win_pend_after = 0;              // batched: deferred idle ticks may be held after it
    long long graph_captures = 0, graph_replays = 0;

    int sticky = 0;
    int stall_test = 0;                  // RANC_TEST_STALL_WAIT (failure-detection tests)
    std::string last_error;
};

namespace ranc {
// Device allocation used by every part of the library.  RANC_FAULT_ALLOC_AFTER=n
// (read by ranc_create) makes the (n+1)-th allocation of that create fail, so
// tests can check that every failure path returns RANC_ENOMEM without leaks.
cudaError_t dev_alloc(void **p, size_t bytes);
void fault_alloc_arm_from_env();
}  // namespace ranc

namespace ranc {
// Implemented in ranc_plain.cu
cudaError_t launch_plain_tick(const PlainArgs &a, cudaStream_t s);
cudaError_t raise_smem_limit(const void *kernel, int bytes);
cudaError_t plain_setup_kernel_attrs(int N, int SW);
cudaError_t launch_plain_windows(const WindowArgs &w, cudaStream_t s);
cudaError_t launch_plain_steps(const PlainArgs &a, int n_ticks, unsigned *bar, cudaStream_t s);
cudaError_t launch_plain_reset(ranc_sim *sim, bool counters);
cudaError_t launch_digest(const int *V, long long n, unsigned long long *out, cudaStream_t s);
// Implemented in ranc_batched.cu
int potential_format_of(const ranc_desc *d);  // kVHalf, kVInt16 or kVInt32 (storage rule of the batched paths)
cudaError_t batched_setup(ranc_sim *sim, const ranc_desc *d, std::string &why);
cudaError_t launch_batched_tick(ranc_sim *sim, const BatchedArgs &a);
cudaError_t launch_batched_reset(ranc_sim *sim, bool counters);
cudaError_t batched_item_ticks(ranc_sim *sim, unsigned long long *host3);  // updated, deferred, active
cudaError_t launch_batched_inputs(ranc_sim *sim, const uint32_t *dev_bits, int n_samples, int n_ticks);
cudaError_t launch_batched_export(ranc_sim *sim, int b0, int nb, int *v_canon, uint32_t *spk_canon,
                                  uint32_t *ring_canon);
cudaError_t launch_batched_import(ranc_sim *sim, const int *v_canon, const uint32_t *spk_canon,
                                  const uint32_t *ring_canon);
cudaError_t batched_export_noalloc(ranc_sim *sim, int b0, int nb, int *v_host, uint32_t *spk_host);
cudaError_t batched_reserve_inputs(ranc_sim *sim, int n_ticks, const void **buffer);
void batched_teardown(ranc_sim *sim);
cudaError_t launch_transpose_inputs(const uint32_t *x, int n_samples, int ticks, int words, int T, uint32_t *inT,
                                    cudaStream_t stream);
// Implemented in ranc_multi.cu (several networks of different core shapes in
// one batched handle, one tick launch for all of them)
bool multi_shape_ok(int axons, int neurons);
int multi_max_stages(int kbmax);
cudaError_t multi_setup(ranc_sim *sim, const ranc_desc *const *descs, int n, std::string &why);
cudaError_t launch_multi_tick(ranc_sim *sim);
cudaError_t launch_multi_reset(ranc_sim *sim, bool counters);
cudaError_t multi_item_ticks(ranc_sim *sim, unsigned long long *host3);  // updated, deferred, active
cudaError_t multi_network_items(ranc_sim *sim, int k, unsigned long long *host2);  // network k: updated, active
int multi_networks(const ranc_sim *sim);
cudaError_t multi_reserve_inputs(ranc_sim *sim, int n_ticks, const void **buffer);
cudaError_t launch_multi_inputs(ranc_sim *sim, const uint32_t *dev_bits, int n_samples, int n_ticks);
cudaError_t launch_multi_export(ranc_sim *sim, int b0, int nb, int *v, uint32_t *spk);
void multi_get_tuning(const ranc_sim *sim, int *stages, int *max_stages, int *cost_item, int *cost_mma, int *cost_slice);
cudaError_t multi_set_tuning(ranc_sim *sim, int stages, int cost_item, int cost_mma, int cost_slice);
void multi_teardown(ranc_sim *sim);
}  // namespace ranc
