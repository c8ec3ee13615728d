/*
 * RANC tick-accurate simulation oracle: a plain, slow, serial C restatement.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  It shares no code,
 * header, table or helper with the CUDA library; the only thing both sides
 * read is the seeded network/input arrays.
 *
 * What it computes follows the paper (GPU-RANC, arXiv 2404.16208):
 *   - Alg. 1 (RANC simulator algorithm): per tick, a scheduler phase over all
 *     cores, routing of the packets of this tick, the neuron block
 *     (core x neuron x axon accumulation, then leak / threshold / reset), and
 *     routing of the spikes produced.
 *   - Sec. II (Background): binary axon x neuron synaptic connections; one
 *     weight per axon type per neuron; LIF neurons; 2-D mesh of cores.
 *   - Sec. III-E (Scheduler): a per-core 2-D boolean array [max tick offset]
 *     x [axons]; at the start of a tick the last tick's row is cleared and the
 *     current-row index advances modulo the maximum offset.
 *   - Sec. III-D (Router): a packet carries the destination core as an offset
 *     and is delivered straight to that core; a spike bit is written into the
 *     destination scheduler row (current + delay).
 *
 * Readings where the paper is silent:
 *   R1 inputs of tick t are written into the row of tick t before the neuron
 *      block (input delay 0);
 *   R2 the scheduler has 16 rows; neuron delays lie in [1, 15];
 *   R3 V <- V + sum(weights of active connected axons) + leak, then compare;
 *   R4 V >= pos_thr spikes (a tie fires) and sets V <- reset;
 *      otherwise V < neg_thr sets V <- neg_thr (mode 0, saturate) or
 *      V <- reset (mode 1);
 *   R5 several packets to one (core, axon, row) are one axon spike (OR);
 *   R6 kind 2 (output bus) counts one event for id = axon field; kind 0 drops
 *      the spike; kind 1 must land on a core (checked, error otherwise);
 *   R7 each sample starts from V = v0, empty scheduler, tick 0;
 *   R8 the potential is computed in 64-bit and must fit int32 (error if not).
 * Parity pinned by: closed-form single-neuron trajectories, hand-worked golden
 * fixtures, delay/row timing, OR merge, packet conservation, a matrix-product
 * identity and brute force against an independent hop-by-hop Python
 * restatement (see the tests).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_ROWS 16 /* scheduler rows (maximum tick offset), reading R2 */

typedef struct {
    int32_t grid_w, grid_h, n_cores, axons, neurons, n_types, neg_mode;
    const int16_t *core_xy;    /* [cores][2] */
    const uint32_t *crossbar;  /* [cores][axons][neurons/32] bit n%32 of word n/32 */
    const uint8_t *axon_type;  /* [cores][axons] */
    const int16_t *weight;     /* [cores][types][neurons] */
    const int32_t *leak, *pos_thr, *neg_thr, *reset, *v0; /* [cores][neurons] */
    const int16_t *dest_dx, *dest_dy;                      /* [cores][neurons] */
    const uint16_t *dest_axon;
    const uint8_t *dest_delay, *dest_kind;
    int32_t n_inputs, n_outputs;
    const int32_t *in_offsets, *in_core, *in_axon;         /* input fan-out CSR */
} oracle_net;

/* Counters per sample: spikes, packets delivered, output events, synaptic
 * events (active axon meets a connection), ticks. */
enum { C_SPIKES = 0, C_PACKETS, C_OUTPUTS, C_SYN, C_TICKS, C_N };

typedef struct {
    int64_t *V;        /* [cores][neurons] membrane potential */
    uint8_t *sched;    /* [cores][ORACLE_ROWS][axons] scheduler SRAM */
    uint8_t *spiked;   /* [cores][neurons] spike flags of the current tick */
    int32_t cur;       /* row index of the current tick (curr_word_index) */
    int32_t *core_at;  /* [grid_h][grid_w] -> core id or -1 */
} oracle_state;

static int synapse(const oracle_net *net, int c, int a, int n)
{
    int words = net->neurons / 32;
    uint32_t w = net->crossbar[((size_t)c * net->axons + a) * words + n / 32];
    return (int)((w >> (n % 32)) & 1u);
}

static uint8_t *row(const oracle_net *net, oracle_state *st, int c, int r)
{
    return st->sched + ((size_t)c * ORACLE_ROWS + r) * net->axons;
}

/* One tick of Alg. 1 for one sample.  in_bits = this tick's input line bits
 * (NULL when the sample has no input at this tick); out_tick, when not NULL,
 * also receives this tick's output-bus events per id. */
static int oracle_tick(const oracle_net *net, oracle_state *st, const uint32_t *in_bits,
                       uint32_t *out_counts, uint32_t *out_tick, uint64_t *cnt, char *err, int errlen)
{
    const int C = net->n_cores, A = net->axons, N = net->neurons;

    /* Scheduler phase (Alg. 1, first per-core loop; Sec. III-E): the row of
     * the last tick is obsolete and cleared, then the index advances. */
    for (int c = 0; c < C; c++)
        memset(row(net, st, c, st->cur), 0, (size_t)A);
    st->cur = (st->cur + 1) % ORACLE_ROWS;

    /* Packets of this tick (Alg. 1, first packet loop): the external input
     * lines, written into the current row (reading R1). */
    if (in_bits) {
        for (int i = 0; i < net->n_inputs; i++) {
            if (!((in_bits[i / 32] >> (i % 32)) & 1u)) continue;
            for (int k = net->in_offsets[i]; k < net->in_offsets[i + 1]; k++)
                row(net, st, net->in_core[k], st->cur)[net->in_axon[k]] = 1;
        }
    }

    /* Neuron block (Alg. 1, core x neuron x axon loops; Sec. II; Sec. III-C). */
    for (int c = 0; c < C; c++) {
        const uint8_t *s = row(net, st, c, st->cur);
        for (int n = 0; n < N; n++) {
            size_t cn = (size_t)c * N + n;
            int64_t acc = 0;
            for (int a = 0; a < A; a++) {
                if (s[a] && synapse(net, c, a, n)) {
                    int k = net->axon_type[(size_t)c * A + a];
                    acc += net->weight[((size_t)c * net->n_types + k) * N + n];
                    cnt[C_SYN]++;
                }
            }
            /* "additional computation / checks": leak, threshold, reset. */
            int64_t v = st->V[cn] + acc + net->leak[cn];
            if (v > INT32_MAX || v < INT32_MIN) {
                snprintf(err, errlen, "potential of core %d neuron %d leaves int32", c, n);
                return -2;
            }
            st->spiked[cn] = 0;
            if (v >= net->pos_thr[cn]) {
                st->spiked[cn] = 1;
                v = net->reset[cn];
            } else if (v < net->neg_thr[cn]) {
                v = (net->neg_mode == 0) ? net->neg_thr[cn] : net->reset[cn];
            }
            st->V[cn] = v;
        }
    }

    /* Routing of the spikes produced (Alg. 1, last core x neuron loop;
     * Sec. III-D): destination computed from the offset, written into the
     * destination scheduler row current + delay. */
    for (int c = 0; c < C; c++) {
        for (int n = 0; n < N; n++) {
            size_t cn = (size_t)c * N + n;
            if (!st->spiked[cn]) continue;
            cnt[C_SPIKES]++;
            int kind = net->dest_kind[cn];
            if (kind == 1) {
                int x = net->core_xy[2 * c] + net->dest_dx[cn];
                int y = net->core_xy[2 * c + 1] + net->dest_dy[cn];
                int d = net->dest_delay[cn];
                int dst = (x >= 0 && x < net->grid_w && y >= 0 && y < net->grid_h)
                              ? st->core_at[y * net->grid_w + x] : -1;
                if (dst < 0 || d < 1 || d >= ORACLE_ROWS || net->dest_axon[cn] >= A) {
                    snprintf(err, errlen, "bad packet from core %d neuron %d", c, n);
                    return -1;
                }
                row(net, st, dst, (st->cur + d) % ORACLE_ROWS)[net->dest_axon[cn]] = 1;
                cnt[C_PACKETS]++;
            } else if (kind == 2) {
                if (net->dest_axon[cn] >= net->n_outputs) {
                    snprintf(err, errlen, "bad output id from core %d neuron %d", c, n);
                    return -1;
                }
                out_counts[net->dest_axon[cn]]++;
                if (out_tick) out_tick[net->dest_axon[cn]]++;
                cnt[C_OUTPUTS]++;
            }
        }
    }
    cnt[C_TICKS]++;
    return 0;
}

/*
 * Run n_samples independent samples for n_ticks ticks each (reading R7).
 *   inputs      [n_samples][t_in][ceil(n_inputs/32)] (ticks >= t_in see no input)
 *   v_final     [n_samples][cores][neurons] potential after the last tick, or NULL
 *   out_counts  [n_samples][n_outputs] output-bus counts over the window
 *   counters    [n_samples][5] (spikes, packets, outputs, synaptic events, ticks)
 *   v_trace     [n_samples][n_ticks][cores][neurons] or NULL
 *   spike_trace [n_samples][n_ticks][cores][neurons] (0/1) or NULL
 *   out_trace   [n_samples][n_ticks][n_outputs] output-bus events of each
 *               tick (the output file of a streamed run, Sec. IV), zeroed by
 *               the caller, or NULL
 *   n_threads   samples are independent; > 1 runs them on OpenMP threads
 * Returns 0, -1 (invalid network) or -2 (potential outside int32); err holds
 * the reason.
 */
int oracle_run(const oracle_net *net, int32_t n_samples, const uint32_t *inputs, int32_t t_in,
               int32_t n_ticks, int32_t *v_final, uint32_t *out_counts, uint64_t *counters,
               int32_t *v_trace, uint8_t *spike_trace, uint32_t *out_trace, int32_t n_threads, char *err,
               int32_t errlen)
{
    const int C = net->n_cores, N = net->neurons;
    const int words = (net->n_inputs + 31) / 32;
    int status = 0;
    err[0] = 0;
    if (net->axons <= 0 || net->neurons <= 0 || net->neurons % 32 != 0 || C <= 0) {
        snprintf(err, errlen, "bad shape");
        return -1;
    }
    int32_t *core_at = (int32_t *)malloc(sizeof(int32_t) * (size_t)net->grid_w * net->grid_h);
    for (int i = 0; i < net->grid_w * net->grid_h; i++) core_at[i] = -1;
    for (int c = 0; c < C; c++) {
        int x = net->core_xy[2 * c], y = net->core_xy[2 * c + 1];
        if (x < 0 || x >= net->grid_w || y < 0 || y >= net->grid_h || core_at[y * net->grid_w + x] >= 0) {
            snprintf(err, errlen, "core %d has a bad or shared grid position", c);
            free(core_at);
            return -1;
        }
        core_at[y * net->grid_w + x] = c;
    }
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
    for (int smp = 0; smp < n_samples; smp++) {
        char lerr[256];
        lerr[0] = 0;
        oracle_state st;
        st.V = (int64_t *)malloc(sizeof(int64_t) * (size_t)C * N);
        st.sched = (uint8_t *)calloc((size_t)C * ORACLE_ROWS * net->axons, 1);
        st.spiked = (uint8_t *)calloc((size_t)C * N, 1);
        st.cur = ORACLE_ROWS - 1; /* so that the first advance selects row 0 */
        st.core_at = core_at;
        for (size_t i = 0; i < (size_t)C * N; i++) st.V[i] = net->v0[i];
        uint64_t *cnt = counters + (size_t)smp * C_N;
        uint32_t *oc = out_counts + (size_t)smp * net->n_outputs;
        memset(cnt, 0, sizeof(uint64_t) * C_N);
        memset(oc, 0, sizeof(uint32_t) * net->n_outputs);
        int rc = 0;
        for (int t = 0; t < n_ticks && rc == 0; t++) {
            const uint32_t *in = (t < t_in) ? inputs + ((size_t)smp * t_in + t) * words : NULL;
            uint32_t *ot = out_trace ? out_trace + ((size_t)smp * n_ticks + t) * net->n_outputs : NULL;
            rc = oracle_tick(net, &st, in, oc, ot, cnt, lerr, sizeof lerr);
            if (rc) break;
            size_t base = ((size_t)smp * n_ticks + t) * C * N;
            for (size_t i = 0; i < (size_t)C * N; i++) {
                if (v_trace) v_trace[base + i] = (int32_t)st.V[i];
                if (spike_trace) spike_trace[base + i] = st.spiked[i];
            }
        }
        if (v_final)
            for (size_t i = 0; i < (size_t)C * N; i++) v_final[(size_t)smp * C * N + i] = (int32_t)st.V[i];
        free(st.V);
        free(st.sched);
        free(st.spiked);
        if (rc) {
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                if (status == 0) {
                    status = rc;
                    snprintf(err, errlen, "sample %d: %s", smp, lerr);
                }
            }
        }
    }
    free(core_at);
    return status;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
