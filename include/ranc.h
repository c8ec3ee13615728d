/*
 * ranc.h - C ABI of the GB300 (sm_103a) RANC tick simulator.
 *
 * The library simulates the per-tick update of every neuromorphic core of a
 * RANC grid (GPU-RANC, arXiv 2404.16208, Alg. 1 and Sec. III): each core
 * reads its active axons from a 16-row scheduler, integrates them through a
 * binary axon x neuron crossbar with one weight per (axon type, neuron), then
 * every neuron applies leak, positive and negative thresholds and reset, and
 * spiking neurons send packets (dx, dy, axon, delay) into row (tick + delay)
 * mod 16 of the destination core's scheduler or count on the output bus.
 *
 * Conventions shared by every entry point
 *   - Return value: RANC_OK (0) or a negative RANC_E* code; the reason is
 *     available from ranc_last_error().  No C++ exception crosses the ABI.
 *   - A CUDA failure (RANC_ECUDA, RANC_ETIMEOUT) makes the handle sticky-failed:
 *     every later call except ranc_reset/ranc_destroy/ranc_last_error returns
 *     RANC_ESTATE until ranc_reset() succeeds.
 *   - All work is ordered on the CUDA stream given to ranc_create (NULL = the
 *     legacy default stream).  Entry points that write host memory synchronise
 *     that stream before returning; the others only enqueue work.
 *   - "host" pointers are ordinary (pageable or pinned) host memory owned by
 *     the caller; "device" pointers are CUDA device memory owned by the
 *     caller.  The library owns every allocation it makes and frees it in
 *     ranc_destroy().  Nothing the caller passes is retained after a call
 *     returns.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *   - Samples are independent copies of the network (a batch); sample b of
 *     every array below is the b-th sample.
 *   - Debug build (libranc_debug.so, compiled with RANC_DEBUG): the tick
 *     kernels check every index they derive from the description before the
 *     global access it addresses (input line and axon of an input entry,
 *     destination core and axon of a packet, output id); a failed check skips
 *     the access and the next synchronising call returns RANC_ECUDA with
 *     "range check failed (site k)" in ranc_last_error.  The environment
 *     variable RANC_DEBUG_PLANT=k, read by ranc_create in that build only,
 *     fails every check of site k on purpose (test use; cleared by ranc_reset).
 */
#ifndef RANC_H
#define RANC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RANC_OK 0
#define RANC_EINVAL (-1)   /* invalid argument or network description */
#define RANC_ENOMEM (-2)   /* device or host allocation failed */
#define RANC_ECUDA (-3)    /* a CUDA runtime call or kernel failed */
#define RANC_ETIMEOUT (-4) /* a bounded device-side wait gave up */
#define RANC_ESTATE (-5)   /* call not valid in the handle's state */

#define RANC_ROWS 16 /* scheduler rows per core: legal delays are 1..15 */

/* Destination kinds of a neuron's spike packet (Sec. III-D). */
enum { RANC_DEST_NONE = 0, RANC_DEST_CORE = 1, RANC_DEST_OUTPUT = 2 };
/* What a potential below the negative threshold becomes. */
enum { RANC_NEG_SATURATE = 0, RANC_NEG_RESET = 1 };
/* Execution path.  PLAIN: one thread per neuron, bit-parallel crossbar
 * integration, any batch.  BATCHED: many samples per core at once, crossbar
 * integration as a tensor-core GEMM (tcgen05) per core; batch is padded
 * internally to a multiple of 128 samples. */
enum { RANC_PATH_PLAIN = 0, RANC_PATH_BATCHED = 1 };
/* Where the buffers of ranc_run_samples live. */
enum { RANC_MEM_HOST = 0, RANC_MEM_DEVICE = 1 };
/* Indices of the counters returned by ranc_read_counters. */
enum {
    RANC_CNT_SPIKES = 0,   /* neurons that fired */
    RANC_CNT_PACKETS = 1,  /* packets delivered to a core (one per kind-core spike) */
    RANC_CNT_OUTPUTS = 2,  /* output-bus events (one per kind-output spike) */
    RANC_CNT_SYNAPTIC = 3, /* (axon, neuron) pairs with an active axon and a connection */
    RANC_CNT_TICKS = 4,    /* sample-ticks simulated (ticks x batch) */
    RANC_N_COUNTERS = 5
};

/* Spike packet of one neuron (Sec. III-D: destination core as an offset,
 * target tick offset and destination axon).  kind = CORE: the packet goes to
 * the core at (x + dx, y + dy), axon `axon`, delay ticks later (1..15).
 * kind = OUTPUT: one output-bus event with id `axon`.  kind = NONE: dropped. */
typedef struct {
    int16_t dx, dy;
    uint16_t axon;
    uint8_t delay, kind;
} ranc_dest;

/* Network / core-parameter description (Sec. II: axons, neurons, synaptic
 * connections, axon types with one weight per type per neuron, CSRAM
 * parameters; Sec. III-B: the per-neuron parameters as one contiguous array).
 * Every array is host memory owned by the caller and read only during
 * ranc_create.  C = n_cores, A = axons, N = neurons, K = n_types.
 *   grid_w, grid_h  mesh size; core_xy[C][2] = (x, y), distinct, in the grid
 *   axons, neurons  multiples of 32, 32..1024
 *   n_types         1..8
 *   weight_bits     2..12: every weight lies in +-(2^(weight_bits-1) - 1)
 *   neg_mode        RANC_NEG_SATURATE or RANC_NEG_RESET
 *   crossbar[C][A][N/32]   synapse (a, n) = bit n%32 of word n/32
 *   axon_type[C][A]        in [0, K)
 *   weight[C][K][N]
 *   leak, pos_thr, neg_thr, reset, v0 [C][N]   (v0 = potential at reset)
 *   dest[C][N]
 *   n_inputs, n_outputs    input lines, output-bus ids (n_outputs >= 1)
 *   in_offsets[n_inputs+1], in_core[nnz], in_axon[nnz]: input line i drives
 *     (in_core[k], in_axon[k]) for k in [in_offsets[i], in_offsets[i+1])
 * The update of a neuron is V <- V + sum of its active connected weights +
 * leak; V >= pos_thr fires and sets V <- reset; otherwise V < neg_thr sets
 * V <- neg_thr (SATURATE) or reset (RESET).  ranc_create rejects a description
 * whose potential could leave int32. */
typedef struct {
    int32_t grid_w, grid_h, n_cores, axons, neurons, n_types, weight_bits, neg_mode;
    const int16_t *core_xy;
    const uint32_t *crossbar;
    const uint8_t *axon_type;
    const int16_t *weight;
    const int32_t *leak, *pos_thr, *neg_thr, *reset, *v0;
    const ranc_dest *dest;
    int32_t n_inputs, n_outputs;
    const int32_t *in_offsets, *in_core, *in_axon;
} ranc_desc;

typedef struct ranc_sim ranc_sim;

/* Validate `desc`, copy it to the device in the layout of `path` and return a
 * handle in *out with every sample at tick 0 (V = v0, empty scheduler, zero
 * outputs and counters).  Sec. III-B/III-E: the CSRAM and scheduler arrays
 * are allocated and copied to the device once.  `cuda_stream` is a
 * cudaStream_t (NULL = default stream) used by every later call.
 * Errors: RANC_EINVAL (bad description, batch < 1, unknown path, no sm_103
 * device for the batched path), RANC_ENOMEM, RANC_ECUDA.  *out is NULL on
 * error. */
int ranc_create(const ranc_desc *desc, int32_t batch, int32_t path, void *cuda_stream, ranc_sim **out);

/* Several networks of different core shapes simulated together in one
 * batched handle: one tick launch updates every core of every network.  The
 * paper motivates GPU simulation by the cost of exploring RANC's configuration
 * space (core sizes, weight widths, axon types, thresholds, delays; Sec. I
 * and Sec. V); a design sweep runs its configurations side by side here.
 * descs[k] (k < n_networks <= 255) is a description as for ranc_create, each
 * with axons a multiple of 64 in [64, 512], neurons a multiple of 128 in
 * [128, 512] and the same neg_mode.  The networks share the batch and the
 * input lines: the handle has max_k n_inputs lines and input line i drives,
 * in every network that has a line i, what that network's fan-out says.
 * Network k's cores and output-bus ids follow those of networks 0 .. k-1:
 * global core = (cores of the networks before) + c, global output id = (ids
 * of the networks before) + id; packets never leave their network.  Every
 * entry point then works on the handle as on a batched one, with these
 * shapes: ranc_read_outputs [batch][sum of n_outputs]; ranc_read_state and
 * ranc_read_sample_state v [samples][P], spikes [samples][P / 32], where
 * P = sum over k of n_cores_k * neurons_k (network k's block of cores at the
 * offset of the networks before, each core's neurons in order);
 * ranc_read_core_counters with global core ranges reads one network's
 * activity.  ranc_run_stream, ranc_save_state, ranc_load_state and
 * ranc_read_sample_state_noalloc return RANC_ESTATE on such a handle.
 * The potentials use the narrowest storage exact for every network (see
 * ranc_potential_format).  Errors: as ranc_create, with the failing
 * network's index in ranc_last_error(NULL). */
int ranc_create_multi(const ranc_desc *const *descs, int32_t n_networks, int32_t batch, void *cuda_stream,
                      ranc_sim **out);

/* Pipeline and split settings of a multi-network handle's tick kernel (the
 * library's own tuning knobs; the paper sweeps CUDA block sizes by hand,
 * Sec. IV).  A work item is one core on one tile of 128 samples; its crossbar
 * product runs as MMAs over 128-neuron slices and 64-axon K-blocks, whose
 * folded weights are copied into a ring of `weight_stages` 16 KB shared-memory
 * stages ahead of the MMAs (2 .. max_weight_stages, which the largest axon
 * count of the handle bounds).  The items of a tick are split over the CTAs by
 * a cost prefix: an item that receives spikes costs cost_item, plus
 * cost_slice per slice, plus cost_mma per (K-block, slice); one that receives
 * none costs 2 * cost_slice per slice.  The defaults (4, 1, 3) fit the
 * kernel's measured per-item, per-slice and per-MMA-group times.  Results
 * do not depend on these settings, only the time does.
 * ranc_set_multi_tuning synchronises the handle's stream, and the next
 * ranc_run_samples call records its window graph again.  Errors:
 * RANC_EINVAL for settings out of range, RANC_ESTATE on a handle made by
 * ranc_create. */
int ranc_set_multi_tuning(ranc_sim *sim, int32_t weight_stages, int32_t cost_item, int32_t cost_mma,
                          int32_t cost_slice);
int ranc_get_multi_tuning(const ranc_sim *sim, int32_t *weight_stages, int32_t *max_weight_stages,
                          int32_t *cost_item, int32_t *cost_mma, int32_t *cost_slice);

/* Replace the input schedule with `bits` (host) [batch][n_ticks][ceil(n_inputs/32)]:
 * line i of input tick j is bit i%32 of word i/32 and is written into the
 * current scheduler row of the cores it drives at tick j counted from the last
 * reset, before the neuron block (Alg. 1, packets of the current tick).
 * Ticks at or beyond n_ticks carry no input.  n_ticks may be 0.  Synchronous. */
int ranc_load_inputs(ranc_sim *sim, const uint32_t *bits, int32_t n_ticks);
/* As ranc_load_inputs, with `bits` in device memory; stream-ordered, no sync. */
int ranc_load_inputs_device(ranc_sim *sim, const uint32_t *bits, int32_t n_ticks);

/* Advance every sample by n_ticks ticks (n_ticks >= 0), each tick a full pass
 * of Alg. 1: scheduler row read and clear, input injection, crossbar
 * integration, leak / threshold / reset, packet delivery and output-bus
 * counting.  Stream-ordered; errors of the enqueued kernels surface at the
 * next synchronising call. */
int ranc_step(ranc_sim *sim, int32_t n_ticks);

/* Output-bus counts since the last reset, [batch][n_outputs] uint32, into host
 * memory (synchronous) or device memory (stream-ordered, no sync). */
int ranc_read_outputs(ranc_sim *sim, uint32_t *counts);
int ranc_read_outputs_device(ranc_sim *sim, uint32_t *counts);

/* Host copies of the state after the last completed tick; each pointer may be
 * NULL.  v [batch][C][N] int32 potentials; spikes [batch][C][N/32] (bit n%32
 * of word n/32 = neuron n fired in the last tick); digest = sum over the flat
 * index i = (b*C + c)*N + n of splitmix64_mix((i << 32) | (uint32)V_i)
 * modulo 2^64, where splitmix64_mix is SplitMix64's output mixing function
 * (order independent, so it is computed on the device).  Synchronous. */
int ranc_read_state(ranc_sim *sim, int32_t *v, uint32_t *spikes, uint64_t *digest);

/* Host copies for samples [b0, b0 + nb) only: v [nb][C][N], spikes
 * [nb][C][N/32], same meaning as in ranc_read_state; either may be NULL.
 * RANC_EINVAL when the range leaves the batch.  Synchronous. */
int ranc_read_sample_state(ranc_sim *sim, int32_t b0, int32_t nb, int32_t *v, uint32_t *spikes);

/* Allocation-free variant of ranc_read_sample_state (the paper has no
 * counterpart; this entry point exists for callers of this library).
 * ranc_read_sample_state on the batched path allocates and frees temporary
 * device buffers on every call.  Some callers cannot do that: applications
 * whose own allocator owns the device memory and forbids allocations outside
 * it, real-time loops that must not allocate (or free, which synchronises the
 * device) after start-up, and callers held to a fixed device-memory budget.
 * This variant converts the state in a fixed scratch array compiled into the
 * library (8 MiB, held by every GPU that loads the library until the process
 * exits) and calls no cudaMalloc, cudaFree or allocating library routine.
 *   - nb * C * N * 4 * (1 + 1/32) bytes must fit in the 8 MiB (512 cores x
 *     256 neurons: at most 15 samples per call); larger ranges return
 *     RANC_EINVAL with the limit in ranc_last_error.
 *   - The first call on a device looks up the scratch array's device address
 *     (once per device); make that first call before any stream capture.
 *     The address is kept for the life of the process: after a reset of the
 *     device's primary context (cudaDeviceReset) it is stale, so do not use
 *     this entry point after one.
 *   - All calls in the process share the one array: calls that overlap on the
 *     GPU (other streams or threads) race.  Every call rewrites the part it
 *     uses, so no call depends on what an earlier call left there.
 * Outputs, meaning and synchronisation are those of ranc_read_sample_state. */
int ranc_read_sample_state_noalloc(ranc_sim *sim, int32_t b0, int32_t nb, int32_t *v, uint32_t *spikes);

/* counters[RANC_N_COUNTERS] summed over the batch since the last ranc_reset
 * (ranc_run_samples keeps accumulating across its windows).  Synchronous. */
int ranc_read_counters(ranc_sim *sim, uint64_t *counters);

/* counters[0..3] (spikes, packets, outputs, synaptic events, as in
 * ranc_read_counters) of the cores core_begin <= c < core_end only, summed
 * over the batch since the last ranc_reset.  A description that combines
 * several independent networks in one grid (a design sweep simulated in one
 * launch per tick) reads each network's activity this way.  RANC_EINVAL for
 * a range outside [0, n_cores].  Synchronous. */
int ranc_read_core_counters(ranc_sim *sim, int32_t core_begin, int32_t core_end, uint64_t *counters);

/* Current tick (counted from the last reset) of every sample. */
int ranc_get_tick(const ranc_sim *sim, int64_t *tick);

/* Back to tick 0: V = v0, empty schedulers, zero outputs, zero counters,
 * spike flags cleared; the input schedule is kept.  Clears a sticky failure
 * when the device is still usable. */
int ranc_reset(ranc_sim *sim);

/* Run sample windows back to back: samples are taken `batch` at a time; each
 * group is reset (counters excepted), given inputs[s][t_in][words] of its
 * samples, stepped `window` ticks, and its output-bus counts are written to
 * counts[s][n_outputs].  A last partial group leaves the unused samples
 * without input and without output.  `mem` says whether `inputs` and `counts`
 * are host (synchronous) or device (stream-ordered) memory.  The paper streams
 * images through one network (Table I) and says nothing of sample boundaries;
 * here every sample starts from V = v0, empty schedulers and tick 0. */
int ranc_run_samples(ranc_sim *sim, const uint32_t *inputs, int32_t n_samples, int32_t t_in, int32_t window,
                     uint32_t *counts, int32_t mem);

/* Streaming, the shape of the paper's MNIST and CIFAR-10 runs (Table I: 10 010
 * ticks, one new image presented per tick and carried through the layers
 * while the next ones enter; the output bus is logged every tick, Sec. IV).
 * Resets the handle as ranc_reset does except for the counters, which keep
 * accumulating; inputs[b][k][words] become the input lines of tick k for
 * k < n_in (no input after); n_ticks ticks are simulated; out_ticks[b][t][id]
 * receives the number of output-bus events of id during tick t (so a stream
 * of frames yields, per frame, the events of the ticks it reaches the bus).
 * ranc_read_outputs afterwards returns the sums over the run.  `mem` says
 * whether `inputs` and `out_ticks` are host (synchronous) or device
 * (stream-ordered) memory.  Plain path: one persistent cooperative launch
 * when the grid fits on the device, per-tick launches otherwise; batched
 * path: per-tick launches (each of the batch's samples is its own stream). */
int ranc_run_stream(ranc_sim *sim, const uint32_t *inputs, int32_t n_in, int32_t n_ticks, uint32_t *out_ticks,
                    int32_t mem);

/* Checkpoint.  ranc_save_state with buf == NULL stores the needed size in *n;
 * otherwise *n must be at least that size and the state after the last
 * completed tick (tick, V, schedulers, outputs, counters, last spikes) is
 * written to buf (host).  ranc_load_state restores a buffer written by a
 * handle with the same description shape, batch and path.  Synchronous. */
int ranc_save_state(ranc_sim *sim, void *buf, size_t *n);
int ranc_load_state(ranc_sim *sim, const void *buf, size_t n);

/* Timing of the tick kernels with CUDA events on the handle's stream (off by
 * default; the events bracket only the kernels that advance ticks).
 * ranc_read_kernel_timing returns their summed duration in milliseconds and
 * the number of ticks they advanced since timing was enabled (one per launch
 * for per-tick kernels; a persistent launch of ranc_run_samples advances
 * window x ceil(n_samples / batch) ticks); synchronous.  A window graph of
 * ranc_run_samples (see ranc_graph_stats) recorded with timing on carries one
 * event pair per group of samples, around that group's `window` tick kernels,
 * so the replays themselves are timed; a replay folds the pairs of the
 * previous one first (synchronising the stream), unless a
 * ranc_read_kernel_timing call in between has done so.  Switching timing on
 * or off makes the next such call record the graph again. */
int ranc_set_kernel_timing(ranc_sim *sim, int32_t enable);
int ranc_read_kernel_timing(ranc_sim *sim, double *total_ms, int64_t *launches);

/* Number of kernels this handle has launched since ranc_create (kernels of a
 * replayed window graph, see ranc_run_samples, included). */
int ranc_launch_count(const ranc_sim *sim, int64_t *launches);

/* CUDA graphs of ranc_run_samples.  On the batched path with device buffers
 * (RANC_MEM_DEVICE) the launch sequence of a call (per group
 * of `batch` samples: reset, input transposition, `window` tick kernels, output
 * copy) depends only on its arguments, so the first call records it as a CUDA
 * graph and later calls with the same inputs, counts, n_samples, t_in and
 * window replay it with one graph launch (a reset that depends on the handle's
 * state runs before it).  The paper launches its kernels one by one from the
 * host every tick (Sec. III); this is the library's own addition.  *captures
 * receives the number of recordings and *replays the number of calls served
 * by a replay.  Errors: RANC_EINVAL if a pointer is NULL. */
int ranc_graph_stats(const ranc_sim *sim, int64_t *captures, int64_t *replays);

/* Work of the batched path's tick kernel.  A work item is one core on one
 * tile of 128 batch slots.  In each tick an item is either updated (its
 * potentials are read and written; the crossbar product runs when its
 * scheduler row or its core's input lines can hold spikes), or, when it
 * receives no spike and every neuron of its core has leak <= 0, reset,
 * theta- and v0 below theta+ and a saturating negative threshold
 * (negative-threshold mode 0), its tick is deferred: such a tick can only
 * take V to max(V + leak, theta-), k of them compose to
 * max(V + k * leak, theta-) (Sec. II, Eq. 1-3 with no input), and that is
 * applied before the item's next update or any state read, so every result
 * is unchanged.  *updated and *deferred receive the item-ticks of each kind
 * since ranc_create or the last ranc_reset (graph replays included).  The
 * call synchronises the handle's stream.  Errors: RANC_EINVAL if a pointer is
 * NULL; RANC_ESTATE on the plain path. */
int ranc_item_ticks(ranc_sim *sim, int64_t *updated, int64_t *deferred);

/* The updated item-ticks of ranc_item_ticks split by what they read: *active
 * receives those whose scheduler row or input lines could hold spikes (the row
 * is read and cleared, the crossbar product runs), *idle those known to
 * receive nothing (no row or input read; dV = 0), *deferred the deferred ones
 * (active + idle = updated).  Same counting period, synchronisation and
 * errors as ranc_item_ticks. */
int ranc_item_classes(ranc_sim *sim, int64_t *active, int64_t *idle, int64_t *deferred);

/* ranc_item_classes for network k of a multi-network handle (ranc_create_multi;
 * its ticks defer nothing): *active and *idle receive that network's
 * item-ticks of each class.  Errors: RANC_EINVAL (NULL pointer, k out of
 * range), RANC_ESTATE on other handles. */
int ranc_network_item_classes(ranc_sim *sim, int32_t k, int64_t *active, int64_t *idle);

/* How the handle stores the membrane potentials in device memory.  The paper
 * makes the potential's bit width a configuration parameter (Sec. III and
 * Sec. V); the library picks, at ranc_create, the narrowest storage that holds
 * every value a neuron can take exactly (the paper gives no overflow rule; the
 * potential is an integer that never wraps):
 *   RANC_POTENTIAL_INT32  int32 (the plain path always; batched otherwise),
 *   RANC_POTENTIAL_INT16  int16: every reachable value, i.e. v0, the reset
 *                         value, theta- and the interval [theta-, theta+ - 1],
 *                         lies in [-32768, 32767],
 *   RANC_POTENTIAL_FP16   IEEE half precision: that range and the range plus
 *                         the leak lie within +-2048, the leak and both
 *                         thresholds lie within [-2047, 2048] (the batched
 *                         tick is then computed on fp16 pairs, still exactly).
 * The choice changes memory traffic only: results are identical in every
 * format.  *format receives one of the values above. */
enum { RANC_POTENTIAL_INT32 = 0, RANC_POTENTIAL_INT16 = 1, RANC_POTENTIAL_FP16 = 2 };
int ranc_potential_format(const ranc_sim *sim, int32_t *format);
/* The storage ranc_create would choose for `desc` on `path` (the same rule),
 * without creating a handle or touching a device: a caller can size memory or
 * group networks by storage before creating anything.  A multi-network handle
 * takes the smallest of its networks' codes (int32 < int16 < fp16).  Errors:
 * RANC_EINVAL for a NULL pointer, an unknown path or a description
 * ranc_create would reject (reason in ranc_last_error(NULL)). */
int ranc_desc_potential_format(const ranc_desc *desc, int32_t path, int32_t *format);

/* Number of device allocations (cudaMalloc calls that succeeded) the library
 * has made in this process since it was loaded, over all handles and threads
 * (the surrogate network of ranc_mlp.h included).  A diagnostic: callers and
 * tests can check that a call allocates nothing.  Errors: RANC_EINVAL if
 * count is NULL. */
int ranc_device_allocations(int64_t *count);

/* Free every device and host resource of the handle.  NULL is a no-op. */
void ranc_destroy(ranc_sim *sim);

/* Reason of the last failure on this handle, or of the last failed
 * ranc_create when sim is NULL.  Never NULL; valid until the next call. */
const char *ranc_last_error(const ranc_sim *sim);

#ifdef __cplusplus
}
#endif
#endif /* RANC_H */
