// Host implementation of the C ABI declared in include/ranc.h.
//
// ranc_create validates the network description, lays it out for the chosen
// path and copies it to the device once (Sec. III-B: the CSRAM becomes one
// contiguous array copied once; Sec. III-E: the schedulers of all cores become
// one array).  Every later call only launches kernels or copies state.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ranc_internal.cuh"
#include "ranc_ptx.cuh"

using namespace ranc;

namespace ranc {
cudaError_t dev_alloc(void **p, size_t bytes);
}

namespace {

constexpr int RANC_ENOTSUP = -100;  // internal: take another code path
thread_local std::string g_create_error;
thread_local long long g_alloc_budget = -1;  // < 0: no fault injection

int fail(ranc_sim *sim, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (sim) {
        sim->last_error = buf;
        if (code == RANC_ECUDA || code == RANC_ETIMEOUT) sim->sticky = 1;
    } else {
        g_create_error = buf;
    }
    return code;
}

#define CUDA_OR_FAIL(sim, expr)                                                                  \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) return fail((sim), RANC_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

#define CHECK_LIVE(sim)                                                                          \
    do {                                                                                         \
        if (!(sim)) return RANC_EINVAL;                                                          \
        if ((sim)->sticky) return fail((sim), RANC_ESTATE, "handle failed earlier: %s; call ranc_reset", \
                                       (sim)->last_error.c_str());                               \
    } while (0)

template <typename T>
cudaError_t dmalloc(T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return dev_alloc(reinterpret_cast<void **>(p), n * sizeof(T));
}

template <typename T>
cudaError_t upload(T **p, const std::vector<T> &h) {
    cudaError_t e = dmalloc(p, h.size());
    if (e != cudaSuccess) return e;
    if (h.empty()) return cudaSuccess;
    return cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

bool bad(std::string &why, const char *fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    why = buf;
    return false;
}

// Checks every rule stated for ranc_desc; fills core_at (grid cell -> core).
bool validate(const ranc_desc *d, int batch, int path, std::vector<int> &core_at, std::string &why) {
    if (!d) return bad(why, "desc is NULL");
    if (batch < 1) return bad(why, "batch must be >= 1 (got %d)", batch);
    if (path != RANC_PATH_PLAIN && path != RANC_PATH_BATCHED) return bad(why, "unknown path %d", path);
    if (d->n_cores < 1) return bad(why, "n_cores must be >= 1");
    if (d->axons < 32 || d->axons > 1024 || d->axons % 32) return bad(why, "axons must be a multiple of 32 in [32, 1024]");
    if (d->neurons < 32 || d->neurons > 1024 || d->neurons % 32)
        return bad(why, "neurons must be a multiple of 32 in [32, 1024]");
    if (d->n_types < 1 || d->n_types > kMaxTypes) return bad(why, "n_types must be in [1, %d]", kMaxTypes);
    if (d->weight_bits < 2 || d->weight_bits > 12) return bad(why, "weight_bits must be in [2, 12]");
    if (d->neg_mode != RANC_NEG_SATURATE && d->neg_mode != RANC_NEG_RESET) return bad(why, "unknown neg_mode");
    if (d->grid_w < 1 || d->grid_h < 1 || (long long)d->grid_w * d->grid_h > (1 << 24)) return bad(why, "bad grid size");
    if (d->n_inputs < 0 || d->n_outputs < 1) return bad(why, "n_inputs must be >= 0 and n_outputs >= 1");
    if (!d->core_xy || !d->crossbar || !d->axon_type || !d->weight || !d->leak || !d->pos_thr || !d->neg_thr ||
        !d->reset || !d->v0 || !d->dest || !d->in_offsets || (d->n_inputs > 0 && (!d->in_core || !d->in_axon)))
        return bad(why, "a required array is NULL");
    const int C = d->n_cores, A = d->axons, N = d->neurons, K = d->n_types;
    core_at.assign((size_t)d->grid_w * d->grid_h, -1);
    for (int c = 0; c < C; c++) {
        const int x = d->core_xy[2 * c], y = d->core_xy[2 * c + 1];
        if (x < 0 || x >= d->grid_w || y < 0 || y >= d->grid_h) return bad(why, "core %d at (%d,%d) is off the grid", c, x, y);
        int &slot = core_at[(size_t)y * d->grid_w + x];
        if (slot >= 0) return bad(why, "cores %d and %d share grid cell (%d,%d)", slot, c, x, y);
        slot = c;
    }
    for (size_t i = 0; i < (size_t)C * A; i++)
        if (d->axon_type[i] >= K) return bad(why, "axon_type[%zu] = %d is not < n_types", i, d->axon_type[i]);
    const int wmax = (1 << (d->weight_bits - 1)) - 1;
    for (size_t i = 0; i < (size_t)C * K * N; i++)
        if (d->weight[i] > wmax || d->weight[i] < -wmax)
            return bad(why, "weight[%zu] = %d is outside +-%d (weight_bits %d)", i, d->weight[i], wmax, d->weight_bits);
    for (int c = 0; c < C; c++) {
        for (int n = 0; n < N; n++) {
            const size_t i = (size_t)c * N + n;
            const ranc_dest &t = d->dest[i];
            if (t.kind == RANC_DEST_NONE) continue;
            if (t.kind == RANC_DEST_OUTPUT) {
                if (t.axon >= d->n_outputs) return bad(why, "core %d neuron %d: output id %d >= n_outputs", c, n, t.axon);
                continue;
            }
            if (t.kind != RANC_DEST_CORE) return bad(why, "core %d neuron %d: unknown destination kind %d", c, n, t.kind);
            if (t.delay < 1 || t.delay >= kRows) return bad(why, "core %d neuron %d: delay %d not in [1, 15]", c, n, t.delay);
            if (t.axon >= A) return bad(why, "core %d neuron %d: destination axon %d >= axons", c, n, t.axon);
            const int x = d->core_xy[2 * c] + t.dx, y = d->core_xy[2 * c + 1] + t.dy;
            if (x < 0 || x >= d->grid_w || y < 0 || y >= d->grid_h || core_at[(size_t)y * d->grid_w + x] < 0)
                return bad(why, "core %d neuron %d: destination (%d,%d) is not a core", c, n, x, y);
        }
        // Potential range (int32 safety): after any tick V lies in
        // [min(neg_thr, reset), max(pos_thr - 1, reset)] or is v0.
        for (int n = 0; n < N; n++) {
            const size_t i = (size_t)c * N + n;
            long long hi = std::max({(long long)d->pos_thr[i] - 1, (long long)d->reset[i], (long long)d->v0[i]});
            long long lo = std::min({(long long)d->neg_thr[i], (long long)d->reset[i], (long long)d->v0[i]});
            long long span = (long long)A * wmax + std::llabs((long long)d->leak[i]);
            if (hi + span > INT32_MAX || lo - span < INT32_MIN)
                return bad(why, "core %d neuron %d: the potential could leave int32", c, n);
        }
    }
    if (d->in_offsets[0] != 0) return bad(why, "in_offsets[0] must be 0");
    for (int i = 0; i < d->n_inputs; i++)
        if (d->in_offsets[i + 1] < d->in_offsets[i]) return bad(why, "in_offsets must be non-decreasing");
    for (int k = 0; k < (d->n_inputs > 0 ? d->in_offsets[d->n_inputs] : 0); k++) {
        if (d->in_core[k] < 0 || d->in_core[k] >= C) return bad(why, "in_core[%d] = %d is not a core", k, d->in_core[k]);
        if (d->in_axon[k] < 0 || d->in_axon[k] >= A) return bad(why, "in_axon[%d] = %d is not an axon", k, d->in_axon[k]);
    }
    return true;
}

void free_all(ranc_sim *s) {
    void *ptrs[] = {s->xbarT, s->wtype, s->axperm, s->wnk, s->prm, s->dst, s->in_ptr, s->in_line, s->in_axon, s->v0,
                    s->V, s->ring, s->spk, s->out, s->cnt, s->inputs, s->err, s->digest, s->stage,
                    s->gbar, s->counts_dev, s->olog_dev};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    batched_teardown(s);
    multi_teardown(s);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    s->ev_pool.clear();
}

// Synchronises the stream and reads the device error word; returns a RANC code.
int check_device_error(ranc_sim *sim) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, sim->err, sizeof(int), cudaMemcpyDeviceToHost, sim->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "kernel failure: %s", cudaGetErrorString(e));
    if (h == kErrTimeout) return fail(sim, RANC_ETIMEOUT, "a device-side wait gave up after %llu ns", kWaitLimitNs);
    if ((h & 0xFF) == kErrBounds) return fail(sim, RANC_ECUDA, "device-side range check failed (site %d)", h >> 8);
    if (h != kErrNone) return fail(sim, RANC_ECUDA, "device error code %d", h);
    return RANC_OK;
}

int sync_and_check(ranc_sim *sim) { return check_device_error(sim); }


int reset_state(ranc_sim *sim, bool counters) {
    cudaError_t e = sim->path == RANC_PATH_PLAIN ? launch_plain_reset(sim, counters)
                    : sim->multi                ? launch_multi_reset(sim, counters)
                                                : launch_batched_reset(sim, counters);
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "reset: %s", cudaGetErrorString(e));
    sim->tick = 0;
    if (counters) sim->ticks_total = 0;
    return RANC_OK;
}

cudaEvent_t next_event(ranc_sim *sim) {
    if (sim->ev_used == (int)sim->ev_pool.size()) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
        sim->ev_pool.push_back(ev);
    }
    return sim->ev_pool[sim->ev_used++];
}

// Folds the recorded event pairs into timed_ms (synchronises the stream):
// the per-launch pairs and, after a timed window-graph launch, the pairs that
// the graph records around each group's tick kernels.
int fold_timing(ranc_sim *sim) {
    if (sim->ev_used == 0 && !sim->win_pending) return RANC_OK;
    CUDA_OR_FAIL(sim, cudaStreamSynchronize(sim->stream));
    if (sim->win_pending) {
        for (size_t i = 0; i + 1 < sim->win_events.size(); i += 2) {
            float ms = 0.f;
            CUDA_OR_FAIL(sim, cudaEventElapsedTime(&ms, sim->win_events[i], sim->win_events[i + 1]));
            sim->timed_ms += ms;
        }
        sim->timed_launches += sim->win_key.window * (long long)sim->win_events.size() / 2;
        sim->win_pending = 0;
    }
    for (int i = 0; i + 1 < sim->ev_used; i += 2) {
        float ms = 0.f;
        CUDA_OR_FAIL(sim, cudaEventElapsedTime(&ms, sim->ev_pool[i], sim->ev_pool[i + 1]));
        sim->timed_ms += ms;
        sim->timed_launches += sim->ev_ticks[i / 2];
    }
    sim->ev_used = 0;
    sim->ev_ticks.clear();
    return RANC_OK;
}

PlainArgs plain_args(const ranc_sim *sim) {
    PlainArgs a{};
    a.C = sim->C; a.A = sim->A; a.N = sim->N; a.K = sim->K; a.AW = sim->A / 32; a.NW = sim->N / 32;
    a.B = sim->B; a.n_valid = sim->n_valid; a.in_words = sim->in_words; a.in_ticks = sim->in_ticks;
    a.n_out = sim->n_outputs; a.neg_mode = sim->neg_mode; a.tick = sim->tick;
    a.xbarT = sim->xbarT; a.wtype = sim->wtype; a.axperm = sim->axperm; a.SW = sim->SW; a.wnk = sim->wnk; a.prm = sim->prm; a.dst = sim->dst;
    a.in_ptr = sim->in_ptr; a.in_line = sim->in_line; a.in_axon = sim->in_axon;
    a.inputs = sim->in_override ? sim->in_override : sim->inputs;
    a.V = (int *)sim->V; a.ring = sim->ring; a.spk = sim->spk; a.out = sim->out; a.cnt = sim->cnt; a.err = sim->err;
    a.stall_test = sim->stall_test;
    a.dbg_plant = sim->dbg_plant;
    a.olog = sim->olog_t; a.olog_stride = sim->olog_stride;
    return a;
}

// Plain path, several ticks without a per-tick output log: one persistent
// cooperative launch (plain_steps_kernel).  RANC_ENOTSUP when it cannot run.
int step_plain_persistent(ranc_sim *sim, int n_ticks) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (sim->timing) {
        if (sim->ev_used + 2 > 4096) {
            int rc = fold_timing(sim);
            if (rc) return rc;
        }
        e0 = next_event(sim);
        e1 = next_event(sim);
        if (!e0 || !e1) return fail(sim, RANC_ECUDA, "cudaEventCreate failed");
        CUDA_OR_FAIL(sim, cudaEventRecord(e0, sim->stream));
    }
    cudaError_t e = launch_plain_steps(plain_args(sim), n_ticks, sim->gbar, sim->stream);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        cudaGetLastError();
        if (sim->timing) sim->ev_used -= 2;
        return RANC_ENOTSUP;
    }
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "persistent tick kernel: %s", cudaGetErrorString(e));
    if (sim->timing) {
        CUDA_OR_FAIL(sim, cudaEventRecord(e1, sim->stream));
        sim->ev_ticks.push_back(n_ticks);
    }
    sim->launches++;
    sim->tick += n_ticks;
    sim->ticks_total += (unsigned long long)sim->n_valid * n_ticks;
    return RANC_OK;
}

int step_ticks(ranc_sim *sim, int n_ticks) {
    if (sim->path == RANC_PATH_PLAIN && n_ticks >= 2 && !sim->olog_t) {
        int rc = step_plain_persistent(sim, n_ticks);
        if (rc != RANC_ENOTSUP) return rc;
    }
    for (int t = 0; t < n_ticks; t++) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (sim->timing) {
            if (sim->ev_used + 2 > 4096) {
                int rc = fold_timing(sim);
                if (rc) return rc;
            }
            e0 = next_event(sim);
            e1 = next_event(sim);
            if (!e0 || !e1) return fail(sim, RANC_ECUDA, "cudaEventCreate failed");
            CUDA_OR_FAIL(sim, cudaEventRecord(e0, sim->stream));
        }
        cudaError_t e;
        if (sim->path == RANC_PATH_PLAIN) {
            e = launch_plain_tick(plain_args(sim), sim->stream);
        } else {
            BatchedArgs a{};
            a.tick = sim->tick;
            e = sim->multi ? launch_multi_tick(sim) : launch_batched_tick(sim, a);
        }
        sim->launches++;
        if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "tick kernel launch: %s", cudaGetErrorString(e));
        if (sim->timing) {
            CUDA_OR_FAIL(sim, cudaEventRecord(e1, sim->stream));
            sim->ev_ticks.push_back(1);
        }
        sim->tick++;
        sim->ticks_total += (unsigned long long)sim->n_valid;
    }
    return RANC_OK;
}

int ensure_inputs(ranc_sim *sim, size_t words) {
    if (words <= sim->inputs_cap) return RANC_OK;
    if (sim->inputs) {
        CUDA_OR_FAIL(sim, cudaStreamSynchronize(sim->stream));
        cudaFree(sim->inputs);
        sim->inputs = nullptr;
        sim->inputs_cap = 0;
    }
    if (dmalloc(&sim->inputs, words) != cudaSuccess) return fail(sim, RANC_ENOMEM, "input buffer of %zu words", words);
    sim->inputs_cap = words;
    return RANC_OK;
}

// Installs inputs for samples [0, n_samples) of the batch (device pointer).
int load_inputs_dev(ranc_sim *sim, const uint32_t *bits, int n_samples, int n_ticks) {
    sim->in_override = nullptr;
    sim->in_ticks = n_ticks;
    sim->n_valid = n_samples;
    if (n_ticks == 0) return RANC_OK;
    if (sim->path == RANC_PATH_PLAIN) {
        const size_t words = (size_t)sim->B * n_ticks * sim->in_words;
        int rc = ensure_inputs(sim, words);
        if (rc) return rc;
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(sim->inputs, bits, (size_t)n_samples * n_ticks * sim->in_words * 4,
                                          cudaMemcpyDeviceToDevice, sim->stream));
        return RANC_OK;
    }
    cudaError_t e = sim->multi ? launch_multi_inputs(sim, bits, n_samples, n_ticks)
                               : launch_batched_inputs(sim, bits, n_samples, n_ticks);
    if (e == cudaErrorMemoryAllocation) return fail(sim, RANC_ENOMEM, "batched input buffers");
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "batched input load: %s", cudaGetErrorString(e));
    return RANC_OK;
}

int ensure_stage(ranc_sim *sim, size_t words) {
    if (words <= sim->stage_cap) return RANC_OK;
    if (sim->stage) {
        CUDA_OR_FAIL(sim, cudaStreamSynchronize(sim->stream));
        cudaFree(sim->stage);
        sim->stage = nullptr;
        sim->stage_cap = 0;
    }
    if (dmalloc(&sim->stage, words) != cudaSuccess) return fail(sim, RANC_ENOMEM, "staging buffer of %zu words", words);
    sim->stage_cap = words;
    return RANC_OK;
}

int load_inputs_host(ranc_sim *sim, const uint32_t *bits, int n_samples, int n_ticks) {
    const size_t words = (size_t)n_samples * n_ticks * sim->in_words;
    if (words == 0) return load_inputs_dev(sim, nullptr, n_samples, 0);
    int rc = ensure_stage(sim, words);
    if (rc) return rc;
    CUDA_OR_FAIL(sim, cudaMemcpyAsync(sim->stage, bits, words * 4, cudaMemcpyHostToDevice, sim->stream));
    rc = load_inputs_dev(sim, sim->stage, n_samples, n_ticks);
    if (rc) return rc;
    CUDA_OR_FAIL(sim, cudaStreamSynchronize(sim->stream));
    return RANC_OK;
}

size_t ring_words(const ranc_sim *s) { return (size_t)s->B * s->C * kRows * (s->A / 32); }

// Canonical state views (plain layout) for read_state / save / load.  For the
// batched path the state is converted by kernels into temporary buffers.
struct Canon {
    int *V = nullptr;
    uint32_t *spk = nullptr, *ring = nullptr;
    bool owned = false;
    ~Canon() {
        if (owned) {
            cudaFree(V);
            cudaFree(spk);
            cudaFree(ring);
        }
    }
};

int canon_view(ranc_sim *sim, Canon &cv, bool need_ring) {
    if (sim->path == RANC_PATH_PLAIN) {
        cv.V = (int *)sim->V;
        cv.spk = sim->spk;
        cv.ring = sim->ring;
        return RANC_OK;
    }
    if (sim->multi && need_ring)
        return fail(sim, RANC_ESTATE, "checkpoints of a multi-network handle are not supported");
    cv.owned = true;
    if (dmalloc(&cv.V, (size_t)sim->B * sim->nps) != cudaSuccess ||
        dmalloc(&cv.spk, (size_t)sim->B * (sim->nps / 32)) != cudaSuccess ||
        (need_ring && dmalloc(&cv.ring, ring_words(sim)) != cudaSuccess))
        return fail(sim, RANC_ENOMEM, "temporary state buffers");
    cudaError_t e = sim->multi ? launch_multi_export(sim, 0, sim->B, cv.V, cv.spk)
                               : launch_batched_export(sim, 0, sim->B, cv.V, cv.spk, need_ring ? cv.ring : nullptr);
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "state export: %s", cudaGetErrorString(e));
    return RANC_OK;
}

struct SaveHeader {
    char magic[8];
    int32_t version, C, A, N, B, path, n_outputs, pad;
    int64_t tick;
    uint64_t ticks_total;
};

size_t save_size(const ranc_sim *s) {
    return sizeof(SaveHeader) + (size_t)s->B * s->C * s->N * 4 + ring_words(s) * 4 + (size_t)s->B * s->n_outputs * 4 +
           (size_t)s->B * s->C * (s->N / 32) * 4 + 4 * 8;
}

// Sums the per-(sample or tile, core) counters rows [..][C][4] over the rows
// whose core lies in [c0, c1).
__global__ void reduce_counters_kernel(const unsigned long long *cnt, long long rows, int C, int c0, int c1,
                                       unsigned long long *out) {
    unsigned long long acc[4] = {0, 0, 0, 0};
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(r % C);
        if (c < c0 || c >= c1) continue;
        for (int j = 0; j < 4; j++) acc[j] += cnt[r * 4 + j];
    }
    for (int j = 0; j < 4; j++) {
        unsigned long long v = acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(out + j, v);
    }
}

int read_counters4(ranc_sim *sim, unsigned long long *h4, int c0 = 0, int c1 = -1) {
    CUDA_OR_FAIL(sim, cudaMemsetAsync(sim->digest, 0, 5 * 8, sim->stream));
    const long long rows = (long long)(sim->cnt_len / 4);
    long long blocks = std::min<long long>((rows + 255) / 256, 1024);
    if (blocks < 1) blocks = 1;
    reduce_counters_kernel<<<(unsigned)blocks, 256, 0, sim->stream>>>(sim->cnt, rows, sim->C, c0, c1 < 0 ? sim->C : c1,
                                                                     sim->digest + 1);
    sim->launches++;
    CUDA_OR_FAIL(sim, cudaGetLastError());
    CUDA_OR_FAIL(sim, cudaMemcpyAsync(h4, sim->digest + 1, 4 * 8, cudaMemcpyDeviceToHost, sim->stream));
    return sync_and_check(sim);
}

}  // namespace

namespace {
std::atomic<long long> g_device_allocations{0};  // successful dev_alloc calls in this process
}

cudaError_t ranc::dev_alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (g_alloc_budget == 0) return cudaErrorMemoryAllocation;
    if (g_alloc_budget > 0) g_alloc_budget--;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_device_allocations.fetch_add(1, std::memory_order_relaxed);
    return e;
}

extern "C" int ranc_device_allocations(int64_t *count) {
    if (!count) return RANC_EINVAL;
    *count = (int64_t)g_device_allocations.load(std::memory_order_relaxed);
    return RANC_OK;
}

void ranc::fault_alloc_arm_from_env() {
    const char *v = getenv("RANC_FAULT_ALLOC_AFTER");
    g_alloc_budget = (v && *v) ? atoll(v) : -1;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" int ranc_create(const ranc_desc *d, int32_t batch, int32_t path, void *cuda_stream, ranc_sim **out) {
    if (!out) return fail(nullptr, RANC_EINVAL, "out is NULL");
    *out = nullptr;
    std::vector<int> core_at;
    std::string why;
    if (!validate(d, batch, path, core_at, why)) return fail(nullptr, RANC_EINVAL, "%s", why.c_str());
    fault_alloc_arm_from_env();
    ranc_sim *sim = new (std::nothrow) ranc_sim();
    if (!sim) return fail(nullptr, RANC_ENOMEM, "host allocation");
    const int C = d->n_cores, A = d->axons, N = d->neurons, K = d->n_types, AW = A / 32;
    sim->C = C; sim->A = A; sim->N = N; sim->K = K; sim->B = batch; sim->path = path; sim->neg_mode = d->neg_mode;
    sim->nps = (long long)C * N;
    sim->grid_w = d->grid_w; sim->grid_h = d->grid_h; sim->n_inputs = d->n_inputs; sim->n_outputs = d->n_outputs;
    sim->in_words = (d->n_inputs + 31) / 32; sim->weight_bits = d->weight_bits;
    sim->stream = static_cast<cudaStream_t>(cuda_stream);
    sim->n_valid = batch;
    {
        const char *st = getenv("RANC_TEST_STALL_WAIT");
        sim->stall_test = (st && *st && *st != '0') ? 1 : 0;
    }
    if (kDebugBuild) {
        const char *pl = getenv("RANC_DEBUG_PLANT");
        sim->dbg_plant = pl ? atoi(pl) : 0;
    }
    auto abort_create = [&](int code, const std::string &msg) {
        g_alloc_budget = -1;
        g_create_error = msg;
        free_all(sim);
        delete sim;
        return code;
    };
    cudaError_t e = cudaGetDevice(&sim->device);
    if (e != cudaSuccess) return abort_create(RANC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));

    // Host-side layout of the constant arrays.
    // Type-sorted axon order of the plain kernels (see PlainArgs::axperm):
    // every type starts at a word boundary, so a core needs sum_k ceil(n_k / 32)
    // words; SW is the largest over the cores.
    int SW = 1;
    for (int c = 0; c < C; c++) {
        std::vector<int> nk(K, 0);
        for (int a = 0; a < A; a++) nk[d->axon_type[(size_t)c * A + a]]++;
        int words = 0;
        for (int k = 0; k < K; k++) words += (nk[k] + 31) / 32;
        SW = std::max(SW, words);
    }
    sim->SW = SW;
    std::vector<uint32_t> xbarT((size_t)C * SW * N, 0u);
    std::vector<int8_t> wtype((size_t)C * SW, (int8_t)-1);
    std::vector<uint16_t> axperm((size_t)C * SW * 32, (uint16_t)0xFFFF);
    std::vector<int16_t> wnk((size_t)C * N * kMaxTypes, 0);
    std::vector<int4> prm((size_t)C * N);
    std::vector<uint2> dst((size_t)C * N);
    const int NWd = N / 32;
    for (int c = 0; c < C; c++) {
        int p = 0;  // next sorted position
        for (int k = 0; k < K; k++) {
            const int p0 = p;
            for (int a = 0; a < A; a++) {
                if (d->axon_type[(size_t)c * A + a] != k) continue;
                axperm[(size_t)c * SW * 32 + p] = (uint16_t)a;
                const uint32_t *src = d->crossbar + ((size_t)c * A + a) * NWd;
                for (int n = 0; n < N; n++)
                    if ((src[n >> 5] >> (n & 31)) & 1u) xbarT[((size_t)c * SW + (p >> 5)) * N + n] |= 1u << (p & 31);
                ++p;
            }
            for (int w = p0 / 32; w < (p + 31) / 32; w++) wtype[(size_t)c * SW + w] = (int8_t)k;
            p = (p + 31) & ~31;
        }
        for (int n = 0; n < N; n++) {
            const size_t i = (size_t)c * N + n;
            for (int k = 0; k < K; k++) wnk[i * kMaxTypes + k] = d->weight[((size_t)c * K + k) * N + n];
            prm[i] = make_int4(d->leak[i], d->pos_thr[i], d->neg_thr[i], d->reset[i]);
            const ranc_dest &t = d->dest[i];
            uint32_t target = 0;
            if (t.kind == RANC_DEST_CORE)
                target = (uint32_t)core_at[(size_t)(d->core_xy[2 * c + 1] + t.dy) * d->grid_w + (d->core_xy[2 * c] + t.dx)];
            else if (t.kind == RANC_DEST_OUTPUT)
                target = t.axon;
            dst[i] = make_uint2(target, (uint32_t)t.axon | ((uint32_t)t.delay << 16) | ((uint32_t)t.kind << 24));
        }
    }
    // Input fan-out regrouped per core: (line, axon) pairs.
    std::vector<int> in_ptr(C + 1, 0), in_line, in_axon;
    const int nnz = d->n_inputs > 0 ? d->in_offsets[d->n_inputs] : 0;
    for (int k = 0; k < nnz; k++) in_ptr[d->in_core[k] + 1]++;
    for (int c = 0; c < C; c++) in_ptr[c + 1] += in_ptr[c];
    in_line.assign(nnz > 0 ? nnz : 1, 0);
    in_axon.assign(nnz > 0 ? nnz : 1, 0);
    {
        std::vector<int> fill(in_ptr.begin(), in_ptr.end() - 1);
        for (int i = 0; i < d->n_inputs; i++)
            for (int k = d->in_offsets[i]; k < d->in_offsets[i + 1]; k++) {
                const int p = fill[d->in_core[k]]++;
                in_line[p] = i;
                in_axon[p] = d->in_axon[k];
            }
    }
    {  // most entries of one core group of the persistent window kernel (its input lists go to shared memory)
        const int G = std::min(kMaxWindowCores, std::max(1, 1024 / N));
        for (int c0 = 0; c0 < C; c0 += G)
            sim->in_group_max = std::max(sim->in_group_max, in_ptr[std::min(C, c0 + G)] - in_ptr[c0]);
    }
    std::vector<int> v0(d->v0, d->v0 + (size_t)C * N);

    if (upload(&sim->xbarT, xbarT) != cudaSuccess || upload(&sim->wtype, wtype) != cudaSuccess ||
        upload(&sim->axperm, axperm) != cudaSuccess ||
        upload(&sim->wnk, wnk) != cudaSuccess || upload(&sim->prm, prm) != cudaSuccess ||
        upload(&sim->dst, dst) != cudaSuccess || upload(&sim->in_ptr, in_ptr) != cudaSuccess ||
        upload(&sim->in_line, in_line) != cudaSuccess || upload(&sim->in_axon, in_axon) != cudaSuccess ||
        upload(&sim->v0, v0) != cudaSuccess || dmalloc(&sim->err, 1) != cudaSuccess ||
        dmalloc(&sim->digest, 8) != cudaSuccess)
        return abort_create(RANC_ENOMEM, "device allocation of the network arrays failed");
    if (cudaMemset(sim->err, 0, sizeof(int)) != cudaSuccess) return abort_create(RANC_ECUDA, "cudaMemset");

    if (path == RANC_PATH_PLAIN) {
        if (dmalloc((int **)&sim->V, (size_t)batch * C * N) != cudaSuccess ||
            dmalloc(&sim->ring, (size_t)batch * C * kRows * AW) != cudaSuccess ||
            dmalloc(&sim->spk, (size_t)batch * C * (N / 32)) != cudaSuccess ||
            dmalloc(&sim->out, (size_t)batch * d->n_outputs) != cudaSuccess ||
            dmalloc(&sim->cnt, (size_t)batch * C * 4) != cudaSuccess || dmalloc(&sim->gbar, 2) != cudaSuccess)
            return abort_create(RANC_ENOMEM, "device allocation of the state arrays failed");
        sim->cnt_len = (size_t)batch * C * 4;
        e = plain_setup_kernel_attrs(N, SW);
        if (e != cudaSuccess) return abort_create(RANC_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    } else {
        e = batched_setup(sim, d, why);
        if (e == cudaErrorInvalidValue) return abort_create(RANC_EINVAL, why);
        if (e == cudaErrorMemoryAllocation) return abort_create(RANC_ENOMEM, why);
        if (e != cudaSuccess) return abort_create(RANC_ECUDA, why + ": " + cudaGetErrorString(e));
    }
    int rc = reset_state(sim, true);
    if (rc == RANC_OK) rc = sync_and_check(sim);
    if (rc != RANC_OK) {
        std::string msg = sim->last_error;
        return abort_create(rc, msg);
    }
    g_alloc_budget = -1;
    *out = sim;
    return RANC_OK;
}

extern "C" int ranc_create_multi(const ranc_desc *const *descs, int32_t n_networks, int32_t batch, void *cuda_stream,
                                 ranc_sim **out) {
    if (!out) return fail(nullptr, RANC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!descs || n_networks < 1 || n_networks > 255) return fail(nullptr, RANC_EINVAL, "n_networks must be in [1, 255]");
    std::string why;
    int n_in = 0, n_out = 0, max_types = 1, max_a = 0, max_n = 0;
    for (int s = 0; s < n_networks; s++) {
        std::vector<int> core_at;
        if (!validate(descs[s], batch, RANC_PATH_BATCHED, core_at, why))
            return fail(nullptr, RANC_EINVAL, "network %d: %s", s, why.c_str());
        const ranc_desc *d = descs[s];
        if (!multi_shape_ok(d->axons, d->neurons))
            return fail(nullptr, RANC_EINVAL,
                        "network %d: a multi-network handle needs axons a multiple of 64 in [64, 512] and neurons a "
                        "multiple of 128 in [128, 512] (got %d x %d)", s, d->axons, d->neurons);
        if (d->neg_mode != descs[0]->neg_mode)
            return fail(nullptr, RANC_EINVAL, "network %d: every network of a multi-network handle needs the same neg_mode", s);
        if ((long long)n_out + d->n_outputs > (1 << 24)) return fail(nullptr, RANC_EINVAL, "too many output ids");
        n_in = std::max(n_in, d->n_inputs);
        n_out += d->n_outputs;
        max_types = std::max(max_types, d->n_types);
        max_a = std::max(max_a, d->axons);
        max_n = std::max(max_n, d->neurons);
    }
    fault_alloc_arm_from_env();
    ranc_sim *sim = new (std::nothrow) ranc_sim();
    if (!sim) return fail(nullptr, RANC_ENOMEM, "host allocation");
    sim->A = max_a; sim->N = max_n; sim->K = max_types; sim->B = batch; sim->path = RANC_PATH_BATCHED;
    sim->neg_mode = descs[0]->neg_mode; sim->n_inputs = n_in; sim->n_outputs = n_out; sim->in_words = (n_in + 31) / 32;
    sim->stream = static_cast<cudaStream_t>(cuda_stream);
    sim->n_valid = batch;
    {
        const char *st = getenv("RANC_TEST_STALL_WAIT");
        sim->stall_test = (st && *st && *st != '0') ? 1 : 0;
    }
    if (kDebugBuild) {
        const char *pl = getenv("RANC_DEBUG_PLANT");
        sim->dbg_plant = pl ? atoi(pl) : 0;
    }
    auto abort_create = [&](int code, const std::string &msg) {
        g_alloc_budget = -1;
        g_create_error = msg;
        free_all(sim);
        delete sim;
        return code;
    };
    cudaError_t e = cudaGetDevice(&sim->device);
    if (e != cudaSuccess) return abort_create(RANC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dmalloc(&sim->err, 1) != cudaSuccess || dmalloc(&sim->digest, 8) != cudaSuccess)
        return abort_create(RANC_ENOMEM, "device allocation failed");
    if (cudaMemset(sim->err, 0, sizeof(int)) != cudaSuccess) return abort_create(RANC_ECUDA, "cudaMemset");
    e = multi_setup(sim, descs, n_networks, why);
    if (e == cudaErrorInvalidValue) return abort_create(RANC_EINVAL, why);
    if (e == cudaErrorMemoryAllocation) return abort_create(RANC_ENOMEM, why);
    if (e != cudaSuccess) return abort_create(RANC_ECUDA, why + ": " + cudaGetErrorString(e));
    int rc = reset_state(sim, true);
    if (rc == RANC_OK) rc = sync_and_check(sim);
    if (rc != RANC_OK) {
        std::string msg = sim->last_error;
        return abort_create(rc, msg);
    }
    g_alloc_budget = -1;
    *out = sim;
    return RANC_OK;
}

extern "C" int ranc_set_multi_tuning(ranc_sim *sim, int32_t weight_stages, int32_t cost_item, int32_t cost_mma,
                                     int32_t cost_slice) {
    CHECK_LIVE(sim);
    if (!sim->multi) return fail(sim, RANC_ESTATE, "the pipeline tuning belongs to multi-network handles");
    int st = 0, mx = 0, ci = 0, cm = 0, cs = 0;
    multi_get_tuning(sim, &st, &mx, &ci, &cm, &cs);
    if (weight_stages < 2 || weight_stages > mx)
        return fail(sim, RANC_EINVAL, "weight stages must be in [2, %d] for this handle (got %d)", mx, weight_stages);
    if (cost_item < 0 || cost_mma < 0 || cost_slice < 1 || cost_item > 1024 || cost_mma > 1024 || cost_slice > 1024)
        return fail(sim, RANC_EINVAL,
                    "split costs must satisfy 0 <= cost_item <= 1024, 0 <= cost_mma <= 1024 and 1 <= cost_slice <= 1024");
    CUDA_OR_FAIL(sim, multi_set_tuning(sim, weight_stages, cost_item, cost_mma, cost_slice));
    if (sim->win_exec) {  // a recorded window graph holds the old launch arguments
        cudaGraphExecDestroy(sim->win_exec);
        sim->win_exec = nullptr;
    }
    return RANC_OK;
}

extern "C" int ranc_get_multi_tuning(const ranc_sim *sim, int32_t *weight_stages, int32_t *max_weight_stages,
                                     int32_t *cost_item, int32_t *cost_mma, int32_t *cost_slice) {
    if (!sim || !weight_stages || !max_weight_stages || !cost_item || !cost_mma || !cost_slice) return RANC_EINVAL;
    if (!sim->multi) return RANC_ESTATE;
    int st = 0, mx = 0, ci = 0, cm = 0, cs = 0;
    multi_get_tuning(sim, &st, &mx, &ci, &cm, &cs);
    *weight_stages = st;
    *max_weight_stages = mx;
    *cost_item = ci;
    *cost_mma = cm;
    *cost_slice = cs;
    return RANC_OK;
}

extern "C" int ranc_load_inputs(ranc_sim *sim, const uint32_t *bits, int32_t n_ticks) {
    CHECK_LIVE(sim);
    if (n_ticks < 0 || (n_ticks > 0 && !bits)) return fail(sim, RANC_EINVAL, "bad input arguments");
    return load_inputs_host(sim, bits, sim->B, n_ticks);
}

extern "C" int ranc_load_inputs_device(ranc_sim *sim, const uint32_t *bits, int32_t n_ticks) {
    CHECK_LIVE(sim);
    if (n_ticks < 0 || (n_ticks > 0 && !bits)) return fail(sim, RANC_EINVAL, "bad input arguments");
    return load_inputs_dev(sim, bits, sim->B, n_ticks);
}

extern "C" int ranc_step(ranc_sim *sim, int32_t n_ticks) {
    CHECK_LIVE(sim);
    if (n_ticks < 0) return fail(sim, RANC_EINVAL, "n_ticks < 0");
    return step_ticks(sim, n_ticks);
}

extern "C" int ranc_read_outputs(ranc_sim *sim, uint32_t *counts) {
    CHECK_LIVE(sim);
    if (!counts) return fail(sim, RANC_EINVAL, "counts is NULL");
    CUDA_OR_FAIL(sim, cudaMemcpyAsync(counts, sim->out, (size_t)sim->B * sim->n_outputs * 4, cudaMemcpyDeviceToHost,
                                      sim->stream));
    return sync_and_check(sim);
}

extern "C" int ranc_read_outputs_device(ranc_sim *sim, uint32_t *counts) {
    CHECK_LIVE(sim);
    if (!counts) return fail(sim, RANC_EINVAL, "counts is NULL");
    CUDA_OR_FAIL(sim, cudaMemcpyAsync(counts, sim->out, (size_t)sim->B * sim->n_outputs * 4,
                                      cudaMemcpyDeviceToDevice, sim->stream));
    return RANC_OK;
}

extern "C" int ranc_read_state(ranc_sim *sim, int32_t *v, uint32_t *spikes, uint64_t *digest) {
    CHECK_LIVE(sim);
    Canon cv;
    int rc = canon_view(sim, cv, false);
    if (rc) return rc;
    const size_t nv = (size_t)sim->B * sim->nps;
    if (v) CUDA_OR_FAIL(sim, cudaMemcpyAsync(v, cv.V, nv * 4, cudaMemcpyDeviceToHost, sim->stream));
    if (spikes)
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(spikes, cv.spk, (size_t)sim->B * (sim->nps / 32) * 4,
                                          cudaMemcpyDeviceToHost, sim->stream));
    if (digest) {
        cudaError_t e = launch_digest(cv.V, (long long)nv, sim->digest, sim->stream);
        sim->launches++;
        if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "digest: %s", cudaGetErrorString(e));
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(digest, sim->digest, 8, cudaMemcpyDeviceToHost, sim->stream));
    }
    return sync_and_check(sim);
}

extern "C" int ranc_read_sample_state(ranc_sim *sim, int32_t b0, int32_t nb, int32_t *v, uint32_t *spikes) {
    CHECK_LIVE(sim);
    if (b0 < 0 || nb < 0 || (long long)b0 + nb > sim->B) return fail(sim, RANC_EINVAL, "sample range outside the batch");
    if (nb == 0) return RANC_OK;
    const size_t per_v = (size_t)sim->nps, per_s = (size_t)sim->nps / 32;
    if (sim->path == RANC_PATH_PLAIN) {
        if (v)
            CUDA_OR_FAIL(sim, cudaMemcpyAsync(v, (int *)sim->V + (size_t)b0 * per_v, (size_t)nb * per_v * 4,
                                              cudaMemcpyDeviceToHost, sim->stream));
        if (spikes)
            CUDA_OR_FAIL(sim, cudaMemcpyAsync(spikes, sim->spk + (size_t)b0 * per_s, (size_t)nb * per_s * 4,
                                              cudaMemcpyDeviceToHost, sim->stream));
        return sync_and_check(sim);
    }
    Canon cv;
    cv.owned = true;
    if (dmalloc(&cv.V, (size_t)nb * per_v) != cudaSuccess || dmalloc(&cv.spk, (size_t)nb * per_s) != cudaSuccess)
        return fail(sim, RANC_ENOMEM, "temporary state buffers");
    cudaError_t e = sim->multi ? launch_multi_export(sim, b0, nb, cv.V, cv.spk)
                               : launch_batched_export(sim, b0, nb, cv.V, cv.spk, nullptr);
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "state export: %s", cudaGetErrorString(e));
    if (v) CUDA_OR_FAIL(sim, cudaMemcpyAsync(v, cv.V, (size_t)nb * per_v * 4, cudaMemcpyDeviceToHost, sim->stream));
    if (spikes)
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(spikes, cv.spk, (size_t)nb * per_s * 4, cudaMemcpyDeviceToHost, sim->stream));
    return sync_and_check(sim);
}

extern "C" int ranc_read_sample_state_noalloc(ranc_sim *sim, int32_t b0, int32_t nb, int32_t *v, uint32_t *spikes) {
    CHECK_LIVE(sim);
    if (b0 < 0 || nb < 0 || (long long)b0 + nb > sim->B) return fail(sim, RANC_EINVAL, "sample range outside the batch");
    if (sim->multi) return fail(sim, RANC_ESTATE, "the allocation-free read does not serve multi-network handles");
    const size_t per_v = (size_t)sim->C * sim->N, per_s = (size_t)sim->C * (sim->N / 32);
    if ((size_t)nb * (per_v + per_s) * 4 > kNoAllocScratchBytes)
        return fail(sim, RANC_EINVAL, "%d samples need %zu bytes of scratch; the allocation-free read holds at most %zu",
                    nb, (size_t)nb * (per_v + per_s) * 4, kNoAllocScratchBytes);
    if (nb == 0) return RANC_OK;
    if (sim->path == RANC_PATH_PLAIN) {  // the state already has the canonical layout: copy it out
        if (v)
            CUDA_OR_FAIL(sim, cudaMemcpyAsync(v, (int *)sim->V + (size_t)b0 * per_v, (size_t)nb * per_v * 4,
                                              cudaMemcpyDeviceToHost, sim->stream));
        if (spikes)
            CUDA_OR_FAIL(sim, cudaMemcpyAsync(spikes, sim->spk + (size_t)b0 * per_s, (size_t)nb * per_s * 4,
                                              cudaMemcpyDeviceToHost, sim->stream));
        return sync_and_check(sim);
    }
    cudaError_t e = batched_export_noalloc(sim, b0, nb, v, spikes);
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "allocation-free state read: %s", cudaGetErrorString(e));
    return sync_and_check(sim);
}

extern "C" int ranc_read_counters(ranc_sim *sim, uint64_t *counters) {
    CHECK_LIVE(sim);
    if (!counters) return fail(sim, RANC_EINVAL, "counters is NULL");
    unsigned long long h4[4];
    int rc = read_counters4(sim, h4);
    if (rc) return rc;
    for (int j = 0; j < 4; j++) counters[j] = h4[j];
    counters[RANC_CNT_TICKS] = sim->ticks_total;
    return RANC_OK;
}

extern "C" int ranc_read_core_counters(ranc_sim *sim, int32_t core_begin, int32_t core_end, uint64_t *counters) {
    CHECK_LIVE(sim);
    if (!counters || core_begin < 0 || core_end < core_begin || core_end > sim->C)
        return fail(sim, RANC_EINVAL, "bad core range [%d, %d) for %d cores", core_begin, core_end, sim->C);
    unsigned long long h4[4];
    int rc = read_counters4(sim, h4, core_begin, core_end);
    if (rc) return rc;
    for (int j = 0; j < 4; j++) counters[j] = h4[j];
    return RANC_OK;
}

extern "C" int ranc_get_tick(const ranc_sim *sim, int64_t *tick) {
    if (!sim || !tick) return RANC_EINVAL;
    *tick = sim->tick;
    return RANC_OK;
}

extern "C" int ranc_reset(ranc_sim *sim) {
    if (!sim) return RANC_EINVAL;
    if ((sim->stall_test || sim->dbg_plant) && sim->win_exec) {  // recorded with the test settings
        cudaStreamSynchronize(sim->stream);
        cudaGraphExecDestroy(sim->win_exec);
        sim->win_exec = nullptr;
    }
    sim->stall_test = 0;  // a stall-test handle runs normally once reset
    sim->dbg_plant = 0;
    if (sim->sticky) {
        cudaError_t e = cudaStreamSynchronize(sim->stream);
        if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "device unusable: %s", cudaGetErrorString(e));
        cudaMemsetAsync(sim->err, 0, sizeof(int), sim->stream);
        sim->sticky = 0;
        sim->ring_all_dirty = 1;  // a failed tick may have left any row written
    }
    sim->ev_used = 0;
    sim->win_pending = 0;
    sim->in_override = nullptr;
    int rc = reset_state(sim, true);
    if (rc) return rc;
    return sync_and_check(sim);
}

// All sample windows of ranc_run_samples in one cooperative launch of the
// persistent plain kernel.  Returns RANC_ENOTSUP when its grid cannot be
// resident at once (the caller then uses per-tick launches).
static int run_windows_persistent(ranc_sim *sim, const uint32_t *inputs, int n_samples, int t_in, int window,
                                  uint32_t *counts, int mem) {
    WindowArgs w{};
    w.G = std::min(kMaxWindowCores, std::max(1, 1024 / sim->N));
    w.in_cap = sim->in_group_max;
    w.n_groups = (sim->C + w.G - 1) / w.G;
    w.n_samples = n_samples;
    w.t_in = t_in;
    w.window = window;
    w.v0 = sim->v0;
    w.bar = sim->gbar;
    const size_t in_words = (size_t)n_samples * t_in * sim->in_words;
    const uint32_t *dev_in = inputs;
    if (mem == RANC_MEM_HOST && in_words > 0) {
        int rc = ensure_stage(sim, in_words);
        if (rc) return rc;
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(sim->stage, inputs, in_words * 4, cudaMemcpyHostToDevice, sim->stream));
        dev_in = sim->stage;
    }
    uint32_t *dev_counts = counts;
    const size_t cwords = (size_t)n_samples * sim->n_outputs;
    if (mem == RANC_MEM_HOST) {
        if (cwords > sim->counts_cap) {
            CUDA_OR_FAIL(sim, cudaStreamSynchronize(sim->stream));
            if (sim->counts_dev) cudaFree(sim->counts_dev);
            sim->counts_dev = nullptr;
            sim->counts_cap = 0;
            if (dmalloc(&sim->counts_dev, cwords) != cudaSuccess) return fail(sim, RANC_ENOMEM, "count buffer");
            sim->counts_cap = cwords;
        }
        dev_counts = sim->counts_dev;
    }
    w.counts = dev_counts;
    PlainArgs &a = w.p;
    a.C = sim->C; a.A = sim->A; a.N = sim->N; a.K = sim->K; a.AW = sim->A / 32; a.NW = sim->N / 32;
    a.B = sim->B; a.n_valid = sim->B; a.in_words = sim->in_words; a.in_ticks = t_in;
    a.n_out = sim->n_outputs; a.neg_mode = sim->neg_mode; a.tick = 0;
    a.xbarT = sim->xbarT; a.wtype = sim->wtype; a.axperm = sim->axperm; a.SW = sim->SW; a.wnk = sim->wnk; a.prm = sim->prm; a.dst = sim->dst;
    a.in_ptr = sim->in_ptr; a.in_line = sim->in_line; a.in_axon = sim->in_axon; a.inputs = dev_in;
    a.V = (int *)sim->V; a.ring = sim->ring; a.spk = sim->spk; a.out = sim->out; a.cnt = sim->cnt; a.err = sim->err;
    a.stall_test = sim->stall_test;
    a.dbg_plant = sim->dbg_plant;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (sim->timing) {
        if (sim->ev_used + 2 > 4096) {
            int rc = fold_timing(sim);
            if (rc) return rc;
        }
        e0 = next_event(sim);
        e1 = next_event(sim);
        if (!e0 || !e1) return fail(sim, RANC_ECUDA, "cudaEventCreate failed");
        CUDA_OR_FAIL(sim, cudaEventRecord(e0, sim->stream));
    }
    cudaError_t e = launch_plain_windows(w, sim->stream);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        cudaGetLastError();
        if (sim->timing) sim->ev_used -= 2;
        return RANC_ENOTSUP;
    }
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "persistent window kernel: %s", cudaGetErrorString(e));
    if (sim->timing) {
        CUDA_OR_FAIL(sim, cudaEventRecord(e1, sim->stream));
        sim->ev_ticks.push_back((long long)window * ((n_samples + sim->B - 1) / sim->B));
    }
    sim->launches++;
    sim->tick = window;
    sim->ticks_total += (unsigned long long)window * n_samples;
    sim->in_override = nullptr;
    sim->in_ticks = 0;
    sim->n_valid = sim->B;
    if (mem == RANC_MEM_HOST) {
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(counts, dev_counts, cwords * 4, cudaMemcpyDeviceToHost, sim->stream));
        return sync_and_check(sim);
    }
    return RANC_OK;
}

// Groups of B samples back to back: (reset, except before the first group),
// inputs, `window` ticks, output counts.  Device buffers only.  `events`
// (NULL, or two per group): recorded as external events right before the
// group's first tick kernel and right after its last one, so that a recorded
// graph carries its own timing of the tick kernels.
static int run_groups_device(ranc_sim *sim, const uint32_t *inputs, int n_samples, int t_in, int window, uint32_t *counts,
                             const cudaEvent_t *events = nullptr) {
    const size_t per = (size_t)t_in * sim->in_words;
    for (int s0 = 0, g = 0; s0 < n_samples; s0 += sim->B, ++g) {
        const int ns = std::min(sim->B, n_samples - s0);
        int rc = s0 > 0 ? reset_state(sim, false) : RANC_OK;
        if (rc) return rc;
        rc = load_inputs_dev(sim, t_in > 0 ? inputs + (size_t)s0 * per : nullptr, ns, t_in);
        if (rc) return rc;
        if (events) CUDA_OR_FAIL(sim, cudaEventRecordWithFlags(events[2 * g], sim->stream, cudaEventRecordExternal));
        rc = step_ticks(sim, window);
        if (rc) return rc;
        if (events) CUDA_OR_FAIL(sim, cudaEventRecordWithFlags(events[2 * g + 1], sim->stream, cudaEventRecordExternal));
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(counts + (size_t)s0 * sim->n_outputs, sim->out, (size_t)ns * sim->n_outputs * 4,
                                          cudaMemcpyDeviceToDevice, sim->stream));
    }
    return RANC_OK;
}

// Batched path, device buffers: every call with the same arguments issues the
// same launch sequence, so it is recorded once as a CUDA graph (on a private
// stream) and replayed by one graph launch afterwards.  The first reset
// depends on the handle's state (which scheduler rows may hold deliveries) and
// runs before the graph; everything after it is fixed by the arguments.
static int run_samples_graph(ranc_sim *sim, const uint32_t *inputs, int n_samples, int t_in, int window, uint32_t *counts) {
    const void *inT = nullptr;
    cudaError_t e = sim->multi ? multi_reserve_inputs(sim, t_in, &inT)  // may allocate: never inside the recording
                               : batched_reserve_inputs(sim, t_in, &inT);
    if (e == cudaErrorMemoryAllocation) return fail(sim, RANC_ENOMEM, "batched input buffers");
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "batched input buffers: %s", cudaGetErrorString(e));
    int rc = reset_state(sim, false);
    if (rc) return rc;
    ranc_sim::WinKey key;
    key.inputs = inputs;
    key.counts = counts;
    key.inT = inT;
    key.n_samples = n_samples;
    key.t_in = t_in;
    key.window = window;
    // With kernel timing on, the recording brackets each group's tick kernels
    // with timing events (folded by the next synchronising timing call); the
    // events of the previous launch are folded first, since a launch records
    // over them.
    const bool timed = sim->timing;
    if (sim->win_pending && (rc = fold_timing(sim)) != RANC_OK) return rc;
    if (sim->win_exec && key == sim->win_key && timed == sim->win_timed) {
        // Host bookkeeping of the recorded sequence, then one launch.
        sim->launches += sim->win_launches;
        sim->ticks_total += sim->win_ticks;
        sim->tick = sim->win_tick_after;
        sim->v_lazy = 0;
        sim->sclock = sim->win_sclock_after;  // the recorded ticks stamp with the recorded clock
        sim->all_active_ticks = 0;
        sim->pend_dirty = sim->win_pend_after;
        CUDA_OR_FAIL(sim, cudaGraphLaunch(sim->win_exec, sim->stream));
        ++sim->graph_replays;
        sim->win_pending = timed ? 1 : 0;
        return RANC_OK;
    }
    if (sim->win_exec) {
        cudaGraphExecDestroy(sim->win_exec);
        sim->win_exec = nullptr;
    }
    if (!sim->cap_stream) CUDA_OR_FAIL(sim, cudaStreamCreateWithFlags(&sim->cap_stream, cudaStreamNonBlocking));
    const size_t n_ev = timed ? 2 * (size_t)((n_samples + sim->B - 1) / sim->B) : 0;
    while (sim->win_events.size() < n_ev) {
        cudaEvent_t ev;
        CUDA_OR_FAIL(sim, cudaEventCreate(&ev));
        sim->win_events.push_back(ev);
    }
    while (sim->win_events.size() > n_ev) {
        cudaEventDestroy(sim->win_events.back());
        sim->win_events.pop_back();
    }
    // The recording reads no device state and the graph runs on the handle's
    // stream, after everything already queued there.
    const cudaStream_t stream = sim->stream;
    const long long l0 = sim->launches;
    const unsigned long long t0 = sim->ticks_total;
    sim->stream = sim->cap_stream;
    e = cudaStreamBeginCapture(sim->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        sim->stream = stream;
        return fail(sim, RANC_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    sim->timing = false;  // the per-launch events of step_ticks are replaced by the recorded ones
    rc = run_groups_device(sim, inputs, n_samples, t_in, window, counts, timed ? sim->win_events.data() : nullptr);
    sim->timing = timed;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(sim->stream, &graph);
    sim->stream = stream;
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return rc ? rc : fail(sim, RANC_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&sim->win_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        sim->win_exec = nullptr;
        return fail(sim, RANC_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    sim->win_key = key;
    sim->win_timed = timed;
    sim->win_launches = sim->launches - l0;
    sim->win_ticks = sim->ticks_total - t0;
    sim->win_tick_after = sim->tick;
    sim->win_sclock_after = sim->sclock;
    sim->win_pend_after = sim->pend_dirty;
    ++sim->graph_captures;
    CUDA_OR_FAIL(sim, cudaGraphLaunch(sim->win_exec, sim->stream));
    sim->win_pending = timed ? 1 : 0;
    return RANC_OK;
}

extern "C" int ranc_item_ticks(ranc_sim *sim, int64_t *updated, int64_t *deferred) {
    CHECK_LIVE(sim);
    if (!updated || !deferred) return RANC_EINVAL;
    if (sim->path != RANC_PATH_BATCHED) return fail(sim, RANC_ESTATE, "item-ticks are counted on the batched path only");
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t e = sim->multi ? multi_item_ticks(sim, h) : batched_item_ticks(sim, h);
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "item-tick counters: %s", cudaGetErrorString(e));
    *updated = (int64_t)h[0];
    *deferred = (int64_t)h[1];
    return RANC_OK;
}

extern "C" int ranc_item_classes(ranc_sim *sim, int64_t *active, int64_t *idle, int64_t *deferred) {
    CHECK_LIVE(sim);
    if (!active || !idle || !deferred) return RANC_EINVAL;
    if (sim->path != RANC_PATH_BATCHED) return fail(sim, RANC_ESTATE, "item-ticks are counted on the batched path only");
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t e = sim->multi ? multi_item_ticks(sim, h) : batched_item_ticks(sim, h);
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "item-tick counters: %s", cudaGetErrorString(e));
    *active = (int64_t)h[2];
    *idle = (int64_t)(h[0] - h[2]);
    *deferred = (int64_t)h[1];
    return RANC_OK;
}

extern "C" int ranc_network_item_classes(ranc_sim *sim, int32_t k, int64_t *active, int64_t *idle) {
    CHECK_LIVE(sim);
    if (!active || !idle) return RANC_EINVAL;
    if (!sim->multi) return fail(sim, RANC_ESTATE, "per-network item-ticks belong to multi-network handles");
    if (k < 0 || k >= multi_networks(sim)) return fail(sim, RANC_EINVAL, "network %d out of range", k);
    unsigned long long h[2] = {0, 0};
    cudaError_t e = multi_network_items(sim, k, h);
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "item-tick counters: %s", cudaGetErrorString(e));
    *active = (int64_t)h[1];
    *idle = (int64_t)(h[0] - h[1]);
    return RANC_OK;
}

extern "C" int ranc_graph_stats(const ranc_sim *sim, int64_t *captures, int64_t *replays) {
    if (!sim || !captures || !replays) return RANC_EINVAL;
    *captures = sim->graph_captures;
    *replays = sim->graph_replays;
    return RANC_OK;
}

extern "C" int ranc_run_samples(ranc_sim *sim, const uint32_t *inputs, int32_t n_samples, int32_t t_in,
                                int32_t window, uint32_t *counts, int32_t mem) {
    CHECK_LIVE(sim);
    if (n_samples < 0 || t_in < 0 || window < 0 || (n_samples > 0 && t_in > 0 && !inputs) ||
        (n_samples > 0 && !counts) || (mem != RANC_MEM_HOST && mem != RANC_MEM_DEVICE))
        return fail(sim, RANC_EINVAL, "bad run_samples arguments");
    const size_t per = (size_t)t_in * sim->in_words;
    if (n_samples == 0) return RANC_OK;
    if (sim->path == RANC_PATH_PLAIN) {
        int rc = run_windows_persistent(sim, inputs, n_samples, t_in, window, counts, mem);
        if (rc != RANC_ENOTSUP) return rc;  // otherwise fall through to per-tick launches
    }
    if (sim->path == RANC_PATH_BATCHED && mem == RANC_MEM_DEVICE) {
        int rc = run_samples_graph(sim, inputs, n_samples, t_in, window, counts);
        sim->in_override = nullptr;
        sim->n_valid = sim->B;
        sim->in_ticks = 0;  // the window inputs are not kept as the handle's schedule
        return rc;
    }
    for (int s0 = 0; s0 < n_samples; s0 += sim->B) {
        const int ns = std::min(sim->B, n_samples - s0);
        int rc = reset_state(sim, false);
        if (rc) return rc;
        if (mem == RANC_MEM_DEVICE && sim->path == RANC_PATH_PLAIN && t_in > 0) {
            sim->in_override = inputs + (size_t)s0 * per;  // read in place, no copy
            sim->in_ticks = t_in;
            sim->n_valid = ns;
        } else if (mem == RANC_MEM_DEVICE) {
            rc = load_inputs_dev(sim, t_in > 0 ? inputs + (size_t)s0 * per : nullptr, ns, t_in);
        } else {
            rc = load_inputs_host(sim, t_in > 0 ? inputs + (size_t)s0 * per : nullptr, ns, t_in);
        }
        if (rc) return rc;
        rc = step_ticks(sim, window);
        if (rc) return rc;
        const size_t ob = (size_t)ns * sim->n_outputs * 4;
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(counts + (size_t)s0 * sim->n_outputs, sim->out, ob,
                                          mem == RANC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                          sim->stream));
    }
    sim->in_override = nullptr;
    sim->n_valid = sim->B;
    sim->in_ticks = 0;  // the window inputs are not kept as the handle's schedule
    if (mem == RANC_MEM_HOST) return sync_and_check(sim);
    return RANC_OK;
}

// Streaming: one persistent cooperative launch of the plain window kernel
// over the whole stream (inputs read from global memory every tick).
static int run_stream_persistent(ranc_sim *sim, const uint32_t *dev_in, int n_in, int n_ticks, uint32_t *dev_log) {
    WindowArgs w{};
    w.G = std::min(kMaxWindowCores, std::max(1, 1024 / sim->N));
    w.in_cap = sim->in_group_max;
    w.n_groups = (sim->C + w.G - 1) / w.G;
    w.n_samples = sim->B;
    w.t_in = n_in;
    w.window = n_ticks;
    w.v0 = sim->v0;
    w.bar = sim->gbar;
    w.counts = nullptr;
    w.stream = 1;
    w.olog = dev_log;
    PlainArgs &a = w.p;
    a.C = sim->C; a.A = sim->A; a.N = sim->N; a.K = sim->K; a.AW = sim->A / 32; a.NW = sim->N / 32;
    a.B = sim->B; a.n_valid = sim->B; a.in_words = sim->in_words; a.in_ticks = n_in;
    a.n_out = sim->n_outputs; a.neg_mode = sim->neg_mode; a.tick = 0;
    a.xbarT = sim->xbarT; a.wtype = sim->wtype; a.axperm = sim->axperm; a.SW = sim->SW; a.wnk = sim->wnk; a.prm = sim->prm; a.dst = sim->dst;
    a.in_ptr = sim->in_ptr; a.in_line = sim->in_line; a.in_axon = sim->in_axon; a.inputs = dev_in;
    a.V = (int *)sim->V; a.ring = sim->ring; a.spk = sim->spk; a.out = sim->out; a.cnt = sim->cnt; a.err = sim->err;
    a.stall_test = sim->stall_test;
    a.dbg_plant = sim->dbg_plant;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (sim->timing) {
        if (sim->ev_used + 2 > 4096) {
            int rc = fold_timing(sim);
            if (rc) return rc;
        }
        e0 = next_event(sim);
        e1 = next_event(sim);
        if (!e0 || !e1) return fail(sim, RANC_ECUDA, "cudaEventCreate failed");
        CUDA_OR_FAIL(sim, cudaEventRecord(e0, sim->stream));
    }
    cudaError_t e = launch_plain_windows(w, sim->stream);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        cudaGetLastError();
        if (sim->timing) sim->ev_used -= 2;
        return RANC_ENOTSUP;
    }
    if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "persistent stream kernel: %s", cudaGetErrorString(e));
    if (sim->timing) {
        CUDA_OR_FAIL(sim, cudaEventRecord(e1, sim->stream));
        sim->ev_ticks.push_back((long long)n_ticks);
    }
    sim->launches++;
    sim->tick = n_ticks;
    sim->ticks_total += (unsigned long long)n_ticks * sim->B;
    sim->in_ticks = 0;
    return RANC_OK;
}

extern "C" int ranc_run_stream(ranc_sim *sim, const uint32_t *inputs, int32_t n_in, int32_t n_ticks,
                               uint32_t *out_ticks, int32_t mem) {
    CHECK_LIVE(sim);
    if (sim->multi) return fail(sim, RANC_ESTATE, "streaming runs of a multi-network handle are not supported");
    if (n_in < 0 || n_ticks < 0 || (n_in > 0 && !inputs) || (n_ticks > 0 && !out_ticks) ||
        (mem != RANC_MEM_HOST && mem != RANC_MEM_DEVICE))
        return fail(sim, RANC_EINVAL, "bad run_stream arguments");
    const size_t lwords = (size_t)sim->B * n_ticks * sim->n_outputs;
    uint32_t *dev_log = out_ticks;
    if (mem == RANC_MEM_HOST && lwords > 0) {
        if (lwords > sim->olog_cap) {
            CUDA_OR_FAIL(sim, cudaStreamSynchronize(sim->stream));
            if (sim->olog_dev) cudaFree(sim->olog_dev);
            sim->olog_dev = nullptr;
            sim->olog_cap = 0;
            if (dmalloc(&sim->olog_dev, lwords) != cudaSuccess) return fail(sim, RANC_ENOMEM, "output log buffer");
            sim->olog_cap = lwords;
        }
        dev_log = sim->olog_dev;
    }
    if (lwords > 0) CUDA_OR_FAIL(sim, cudaMemsetAsync(dev_log, 0, lwords * 4, sim->stream));
    int rc = RANC_ENOTSUP;
    if (sim->path == RANC_PATH_PLAIN) {
        // Inputs on the device as [B][n_in][words] for the persistent kernel.
        const size_t in_words = (size_t)sim->B * n_in * sim->in_words;
        const uint32_t *dev_in = inputs;
        if (mem == RANC_MEM_HOST && in_words > 0) {
            rc = ensure_stage(sim, in_words);
            if (rc) return rc;
            CUDA_OR_FAIL(sim, cudaMemcpyAsync(sim->stage, inputs, in_words * 4, cudaMemcpyHostToDevice, sim->stream));
            dev_in = sim->stage;
        }
        rc = run_stream_persistent(sim, dev_in, n_in, n_ticks, dev_log);
        if (rc != RANC_OK && rc != RANC_ENOTSUP) return rc;
    }
    if (rc == RANC_ENOTSUP) {  // per-tick launches: reset, input schedule, one log slot per tick
        rc = reset_state(sim, false);
        if (rc) return rc;
        rc = mem == RANC_MEM_DEVICE ? load_inputs_dev(sim, n_in > 0 ? inputs : nullptr, sim->B, n_in)
                                    : load_inputs_host(sim, n_in > 0 ? inputs : nullptr, sim->B, n_in);
        if (rc) return rc;
        sim->olog_stride = (long long)n_ticks * sim->n_outputs;
        for (int t = 0; t < n_ticks && rc == RANC_OK; t++) {
            sim->olog_t = dev_log + (size_t)t * sim->n_outputs;
            rc = step_ticks(sim, 1);
        }
        sim->olog_t = nullptr;
        sim->olog_stride = 0;
        sim->in_ticks = 0;  // the stream's inputs are not kept as the handle's schedule
        if (rc) return rc;
    }
    if (mem == RANC_MEM_HOST) {
        if (lwords > 0)
            CUDA_OR_FAIL(sim, cudaMemcpyAsync(out_ticks, dev_log, lwords * 4, cudaMemcpyDeviceToHost, sim->stream));
        return sync_and_check(sim);
    }
    return RANC_OK;
}

extern "C" int ranc_save_state(ranc_sim *sim, void *buf, size_t *n) {
    CHECK_LIVE(sim);
    if (sim->multi) return fail(sim, RANC_ESTATE, "checkpoints of a multi-network handle are not supported");
    if (!n) return fail(sim, RANC_EINVAL, "n is NULL");
    const size_t need = save_size(sim);
    if (!buf) {
        *n = need;
        return RANC_OK;
    }
    if (*n < need) return fail(sim, RANC_EINVAL, "buffer of %zu bytes < %zu", *n, need);
    Canon cv;
    int rc = canon_view(sim, cv, true);
    if (rc) return rc;
    SaveHeader h{};
    memcpy(h.magic, "RANCSTA", 8);
    h.version = 1; h.C = sim->C; h.A = sim->A; h.N = sim->N; h.B = sim->B; h.path = sim->path;
    h.n_outputs = sim->n_outputs; h.tick = sim->tick; h.ticks_total = sim->ticks_total;
    char *p = static_cast<char *>(buf);
    memcpy(p, &h, sizeof h);
    p += sizeof h;
    const size_t nv = (size_t)sim->B * sim->C * sim->N * 4, nr = ring_words(sim) * 4,
                 no = (size_t)sim->B * sim->n_outputs * 4, ns = (size_t)sim->B * sim->C * (sim->N / 32) * 4;
    CUDA_OR_FAIL(sim, cudaMemcpyAsync(p, cv.V, nv, cudaMemcpyDeviceToHost, sim->stream));
    p += nv;
    CUDA_OR_FAIL(sim, cudaMemcpyAsync(p, cv.ring, nr, cudaMemcpyDeviceToHost, sim->stream));
    p += nr;
    CUDA_OR_FAIL(sim, cudaMemcpyAsync(p, sim->out, no, cudaMemcpyDeviceToHost, sim->stream));
    p += no;
    CUDA_OR_FAIL(sim, cudaMemcpyAsync(p, cv.spk, ns, cudaMemcpyDeviceToHost, sim->stream));
    p += ns;
    unsigned long long h4[4];
    rc = read_counters4(sim, h4);
    if (rc) return rc;
    memcpy(p, h4, sizeof h4);
    *n = need;
    return RANC_OK;
}

__global__ void load_counters_kernel(unsigned long long *cnt, unsigned long long c0, unsigned long long c1,
                                     unsigned long long c2, unsigned long long c3) {
    cnt[0] = c0;
    cnt[1] = c1;
    cnt[2] = c2;
    cnt[3] = c3;
}

extern "C" int ranc_load_state(ranc_sim *sim, const void *buf, size_t n) {
    CHECK_LIVE(sim);
    if (sim->multi) return fail(sim, RANC_ESTATE, "checkpoints of a multi-network handle are not supported");
    if (!buf || n < save_size(sim)) return fail(sim, RANC_EINVAL, "state buffer too small");
    SaveHeader h;
    memcpy(&h, buf, sizeof h);
    if (memcmp(h.magic, "RANCSTA", 8) != 0 || h.version != 1 || h.C != sim->C || h.A != sim->A || h.N != sim->N ||
        h.B != sim->B || h.path != sim->path || h.n_outputs != sim->n_outputs)
        return fail(sim, RANC_EINVAL, "state buffer does not match this handle");
    const char *p = static_cast<const char *>(buf) + sizeof h;
    const size_t nv = (size_t)sim->B * sim->C * sim->N * 4, nr = ring_words(sim) * 4,
                 no = (size_t)sim->B * sim->n_outputs * 4, ns = (size_t)sim->B * sim->C * (sim->N / 32) * 4;
    unsigned long long h4[4];
    memcpy(h4, p + nv + nr + no + ns, sizeof h4);
    if (sim->path == RANC_PATH_PLAIN) {
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(sim->V, p, nv, cudaMemcpyHostToDevice, sim->stream));
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(sim->ring, p + nv, nr, cudaMemcpyHostToDevice, sim->stream));
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(sim->spk, p + nv + nr + no, ns, cudaMemcpyHostToDevice, sim->stream));
    } else {
        Canon cv;
        cv.owned = true;
        if (dmalloc(&cv.V, nv / 4) != cudaSuccess || dmalloc(&cv.ring, nr / 4) != cudaSuccess ||
            dmalloc(&cv.spk, ns / 4) != cudaSuccess)
            return fail(sim, RANC_ENOMEM, "temporary state buffers");
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(cv.V, p, nv, cudaMemcpyHostToDevice, sim->stream));
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(cv.ring, p + nv, nr, cudaMemcpyHostToDevice, sim->stream));
        CUDA_OR_FAIL(sim, cudaMemcpyAsync(cv.spk, p + nv + nr + no, ns, cudaMemcpyHostToDevice, sim->stream));
        cudaError_t e = launch_batched_import(sim, cv.V, cv.spk, cv.ring);
        if (e != cudaSuccess) return fail(sim, RANC_ECUDA, "state import: %s", cudaGetErrorString(e));
        CUDA_OR_FAIL(sim, cudaStreamSynchronize(sim->stream));
    }
    CUDA_OR_FAIL(sim, cudaMemcpyAsync(sim->out, p + nv + nr, no, cudaMemcpyHostToDevice, sim->stream));
    // The partial counters collapse into row 0.
    CUDA_OR_FAIL(sim, cudaMemsetAsync(sim->cnt, 0, sim->cnt_len * 8, sim->stream));
    load_counters_kernel<<<1, 1, 0, sim->stream>>>(sim->cnt, h4[0], h4[1], h4[2], h4[3]);
    sim->launches++;
    CUDA_OR_FAIL(sim, cudaGetLastError());
    sim->tick = h.tick;
    sim->ticks_total = h.ticks_total;
    return sync_and_check(sim);
}

extern "C" int ranc_set_kernel_timing(ranc_sim *sim, int32_t enable) {
    CHECK_LIVE(sim);
    int rc = fold_timing(sim);
    if (rc) return rc;
    sim->timing = enable != 0;
    sim->timed_ms = 0.0;
    sim->timed_launches = 0;
    return RANC_OK;
}

extern "C" int ranc_read_kernel_timing(ranc_sim *sim, double *total_ms, int64_t *launches) {
    CHECK_LIVE(sim);
    int rc = fold_timing(sim);
    if (rc) return rc;
    if (total_ms) *total_ms = sim->timed_ms;
    if (launches) *launches = sim->timed_launches;
    return RANC_OK;
}

extern "C" int ranc_launch_count(const ranc_sim *sim, int64_t *launches) {
    if (!sim || !launches) return RANC_EINVAL;
    *launches = sim->launches;
    return RANC_OK;
}

extern "C" int ranc_potential_format(const ranc_sim *sim, int32_t *format) {
    if (!sim || !format) return RANC_EINVAL;
    static_assert(RANC_POTENTIAL_INT32 == kVInt32 && RANC_POTENTIAL_INT16 == kVInt16 && RANC_POTENTIAL_FP16 == kVHalf,
                  "storage codes");
    *format = sim->path == RANC_PATH_PLAIN ? RANC_POTENTIAL_INT32 : sim->vmode;
    return RANC_OK;
}

extern "C" int ranc_desc_potential_format(const ranc_desc *desc, int32_t path, int32_t *format) {
    if (!desc || !format || (path != RANC_PATH_PLAIN && path != RANC_PATH_BATCHED)) return RANC_EINVAL;
    std::vector<int> core_at;
    std::string why;
    if (!validate(desc, 1, path, core_at, why)) return fail(nullptr, RANC_EINVAL, "%s", why.c_str());
    *format = path == RANC_PATH_PLAIN ? RANC_POTENTIAL_INT32 : potential_format_of(desc);
    return RANC_OK;
}

extern "C" void ranc_destroy(ranc_sim *sim) {
    if (!sim) return;
    cudaStreamSynchronize(sim->stream);
    if (sim->win_exec) cudaGraphExecDestroy(sim->win_exec);
    for (cudaEvent_t ev : sim->win_events) cudaEventDestroy(ev);
    if (sim->cap_stream) cudaStreamDestroy(sim->cap_stream);
    free_all(sim);
    delete sim;
}

extern "C" const char *ranc_last_error(const ranc_sim *sim) {
    if (!sim) return g_create_error.c_str();
    return sim->last_error.c_str();
}
