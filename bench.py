"""Benchmark of the RANC hot path on one GB300 (JSON line on stdout).

Workload: the MNIST-shaped 512-core, 3-layer net (32 x 16 grid, 256 axons x
256 neurons per core, 4 axon types, 9-bit weights, delays 1..4), seeded
synthetic 28x28 inputs rate-coded over 16 ticks, 24-tick sample windows.

* batched leg (headline): 4096 samples per step in one batched handle
  (tensor-core crossbar integration), inputs resident on the device;
* plain leg: 10,000 samples per step, one sample at a time (batch 1), the
  paper's execution model;
* e2e: the batched step through the C ABI with host buffers (inputs copied in
  and output counts copied out inside the timed region);
* roofline: the dominant tick kernel, timed with CUDA events on its stream;
* cpu_baseline: the CPU oracle on a bounded sample of the same workload.

``--impl reference`` times the CPU oracle alone (the reference arm of this
project) and prints its own line.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "synaptic events/sec and samples/sec (512-core net), batched vs plain, bit-exact"
T_IN, WINDOW = 16, 24
PLAIN_SAMPLES, BATCH_SAMPLES = 10000, 4096
L2_FLUSH_BYTES = 512 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], bf16_tflops=d["bf16_tflops"],
                    bf16_tflops_sustained=d.get("bf16_tflops_sustained", d["bf16_tflops"]), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, source="fallback")


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws, int(os.environ.get("LOCAL_RANK", "0"))


def make_workload(first_sample, n_samples):
    import ranc_workloads as W
    net = W.mnist_512core()
    x = W.rate_coded_inputs(net.meta["seed"], n_samples, T_IN, net.n_inputs, net.meta["p_in"],
                            first_sample=first_sample)
    return net, x


def oracle_rate(net, x_all, budget_s=12.0, threads=None):
    """Times the CPU oracle on a bounded prefix of the samples."""
    import oracle
    oracle.build()
    threads = threads or os.cpu_count() or 1
    n = max(1, min(threads, x_all.shape[0]))
    t0 = time.perf_counter()
    r = oracle.run(net, x_all[:n], WINDOW, n_threads=threads)
    dt = time.perf_counter() - t0
    total_s, total_n, events = dt, n, int(r["counters"][:, 3].sum())
    more = int(min(x_all.shape[0] - n, max(0, (budget_s - dt) / max(dt / n, 1e-9))))
    if more > 0:
        t0 = time.perf_counter()
        r = oracle.run(net, x_all[n:n + more], WINDOW, n_threads=threads)
        total_s += time.perf_counter() - t0
        total_n += more
        events += int(r["counters"][:, 3].sum())
    return dict(samples=total_n, seconds=total_s, samples_per_s=total_n / total_s, events_per_s=events / total_s,
                threads=threads)


def flush_l2(buf):
    buf.add_(1)


def bench_plain(ranc, torch, net, dx, n_samples, steps, warmup, flush):
    """Plain path, batch 1: every sample's window back to back on the device."""
    sim = ranc.Sim(net, 1, ranc.RANC_PATH_PLAIN)
    dout = torch.zeros((n_samples, net.n_outputs), dtype=torch.int32, device="cuda")
    run = lambda: ranc.ranc_run_samples(sim.h, dx.data_ptr(), n_samples, T_IN, WINDOW, dout.data_ptr(),
                                        ranc.RANC_MEM_DEVICE)
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    ranc.ranc_reset(sim.h)
    l0 = ranc.ranc_launch_count(sim.h)
    ms = 0.0
    for _ in range(steps):
        flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    launches = ranc.ranc_launch_count(sim.h) - l0
    cnt = ranc.ranc_read_counters(sim.h)
    # Per-kernel durations (CUDA events around each tick kernel on the
    # handle's stream), taken on a separate pass so the events do not slow
    # the timed steps.
    ranc.ranc_set_kernel_timing(sim.h, True)
    ranc.ranc_run_samples(sim.h, dx.data_ptr(), min(n_samples, 500), T_IN, WINDOW, dout.data_ptr(),
                          ranc.RANC_MEM_DEVICE)
    kms, kn = ranc.ranc_read_kernel_timing(sim.h)
    ranc.ranc_set_kernel_timing(sim.h, False)
    sim.close()
    return dict(ms=ms, samples=n_samples * steps, events=int(cnt[3]), launches=launches, kernel_ms=kms,
                kernel_launches=kn, counts=dout.cpu().numpy())


def plain_bytes_per_core_tick(net):
    """Algorithmic bytes one core-tick of the plain kernel must move."""
    A, N, K = net.axons, net.neurons, net.n_types
    return (N * A // 8          # crossbar bits
            + N * 8             # V read + write (int32)
            + N * 16            # leak, pos_thr, neg_thr, reset
            + N * 2 * K         # weights (int16)
            + N * 8             # destination word
            + 2 * A // 8        # scheduler row read + clear
            + K * A // 8        # axon-type masks
            + N // 8)           # spike bitmap


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--plain-samples", type=int, default=PLAIN_SAMPLES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank, ws, local = dist_env()

    if args.impl == "reference":
        if rank != 0:
            return
        net, x = make_workload(0, 512)
        steps_ms, tot_n, tot_ev = [], 0, 0.0
        import oracle
        oracle.build()
        thr = os.cpu_count() or 1
        for i in range(args.warmup + args.steps):
            xs = x[(i * thr) % 256:(i * thr) % 256 + thr]
            t0 = time.perf_counter()
            r = oracle.run(net, xs, WINDOW, n_threads=thr)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                steps_ms.append(dt * 1e3)
                tot_n += xs.shape[0]
                tot_ev += float(r["counters"][:, 3].sum())
        sec = sum(steps_ms) / 1e3
        val = tot_n / sec
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": val, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(steps_ms) / len(steps_ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "synaptic_events_per_sec": tot_ev / sec,
            "config": {"workload": "mnist-shaped 512-core net, 24-tick windows, CPU oracle",
                       "samples_per_step": thr},
            "cpu_baseline": {"value": val, "unit": "samples/s", "cores": thr, "kind": "oracle",
                             "sample": f"{thr} samples of the 512-core workload per step"},
            "e2e": {"value": val, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    import torch
    from paper_2404_16208_gb300 import build_library
    build_library()
    from paper_2404_16208_gb300 import ranc

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    pk = peaks()
    # Samples are independent: each rank takes its own slice (no data-path collective).
    first = rank * args.plain_samples
    net, x = make_workload(first, args.plain_samples)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        pr = bench_plain(ranc, torch, net, dx, args.plain_samples, args.steps, args.warmup, flush)
    t_plain = torch.tensor([pr["ms"]], device="cuda")
    if ws > 1:
        dist.all_reduce(t_plain, op=dist.ReduceOp.MAX)
    ms_plain = float(t_plain.item())

    # roofline of the dominant kernel (plain tick kernel for now)
    kavg = pr["kernel_ms"] / max(pr["kernel_launches"], 1)
    bytes_launch = plain_bytes_per_core_tick(net) * net.n_cores
    achieved = bytes_launch / (kavg * 1e-3) / 1e9
    roof = {"kernel": "plain_tick_kernel", "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
            "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": None,
            "peak_source": pk["source"], "avg_launch_us": kavg * 1e3, "bytes_per_launch": bytes_launch}

    # e2e: host buffers through the C ABI (plain leg until the batched path lands)
    e2e_n = min(args.plain_samples, 2000)
    xh = torch.from_numpy(x[:e2e_n].copy()).pin_memory().numpy()
    ch = torch.zeros((e2e_n, net.n_outputs), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    sim = ranc.Sim(net, 1, ranc.RANC_PATH_PLAIN)
    ranc.ranc_run_samples(sim.h, xh, e2e_n, T_IN, WINDOW, ch)
    t0 = time.perf_counter()
    ranc.ranc_run_samples(sim.h, xh, e2e_n, T_IN, WINDOW, ch)
    e2e_s = time.perf_counter() - t0
    sim.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cr = oracle_rate(net, x[:256])
        cpu = {"value": cr["samples_per_s"], "unit": "samples/s", "cores": cr["threads"], "kind": "oracle",
               "sample": f"{cr['samples']} samples of the 512-core workload ({cr['seconds']:.1f} s)",
               "synaptic_events_per_sec": cr["events_per_s"]}

    samples_total = pr["samples"] * ws
    val = samples_total / (ms_plain * 1e-3)
    line = {
        "metric": METRIC, "value": val, "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_plain / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "synaptic_events_per_sec": pr["events"] * ws / (ms_plain * 1e-3),
        "config": {"workload": f"mnist-shaped 512-core net, plain path, batch 1, {args.plain_samples} samples "
                               f"x {WINDOW} ticks per step", "l2": "flushed between timed steps (512 MiB write)",
                   "path": "plain"},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": e2e_n / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": int(xh.nbytes),
                "d2h_bytes_per_step": int(ch.nbytes)},
        "clocks": clk.summary(), "gpu_launches": int(pr["launches"]),
    }
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
